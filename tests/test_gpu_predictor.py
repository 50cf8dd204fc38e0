"""The learned slice predictor on the GPU: kernels against the oracle, labels, training, and its gain."""
import numpy as np
import pytest
import torch

from oracle import df_oracle as O
from oracle import mlp_oracle as M
from paper_2601_08077_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def df():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_08077_gb300 import build, df as dfmod
    build.build_all()
    return dfmod


def test_mlp_forward_and_gradients_match_oracle(df):
    rng = np.random.default_rng(5)
    theta = (M.init_params(9) + 0.05 * rng.standard_normal(M.N_PARAMS)).astype(np.float32)
    X = rng.standard_normal((37, 16)).astype(np.float32)
    y = rng.integers(0, 8, size=37)
    net = df.MLP(theta)
    Xg = torch.from_numpy(X).cuda()
    yg = torch.from_numpy(y.astype(np.int32)).cuda()
    probs = net.forward(Xg).cpu().numpy()
    ref_p, _ = M.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(probs - ref_p)) < 1e-5
    g, loss = net.gradients(Xg, yg)
    g_ref = M.gradients(theta.astype(np.float64), X.astype(np.float64), y)
    assert abs(loss - M.loss(theta.astype(np.float64), X.astype(np.float64), y)) < 1e-5
    assert np.max(np.abs(g - g_ref)) <= 1e-5 + 1e-4 * np.max(np.abs(g_ref))


def test_adam_steps_match_oracle(df):
    """Three df_mlp_train_step calls against the oracle's Adam (beta 0.9 / 0.999, bias
    correction) on the oracle's FP64 gradients, element by element.  The first update is
    lr g / (|g| + eps) ~ lr sign(g), so an element whose gradient is within the FP32
    gradient error of zero may take either sign: those get a bound of 2 lr per step, the
    rest must agree to 2 % of lr per step."""
    rng = np.random.default_rng(11)
    theta0 = (M.init_params(4) + 0.05 * rng.standard_normal(M.N_PARAMS)).astype(np.float32)
    X = rng.standard_normal((96, 16)).astype(np.float32)
    y = rng.integers(0, 8, size=96)
    net = df.MLP(theta0)
    Xg = torch.from_numpy(X).cuda()
    yg = torch.from_numpy(y.astype(np.int32)).cuda()
    lr = 1e-3
    th = theta0.astype(np.float64)
    m = np.zeros(M.N_PARAMS)
    v = np.zeros(M.N_PARAMS)
    gmin = np.full(M.N_PARAMS, np.inf)
    for t in (1, 2, 3):
        g = M.gradients(th, X.astype(np.float64), y)
        gmin = np.minimum(gmin, np.abs(g))
        th, m, v = M.adam_step(th, g, m, v, t, lr)
        net.train_step(Xg, yg, lr)
        got = net.get_params().astype(np.float64)
        sure = gmin > 1e-3 * np.max(np.abs(g))
        diff = np.abs(got - th)
        assert sure.sum() > 0.5 * M.N_PARAMS
        assert np.max(diff[sure]) <= 0.02 * lr * t + 1e-7
        assert np.max(diff) <= 2 * lr * t + 1e-7
    # the parameters really moved by about lr per step (no update lost)
    moved = np.abs(net.get_params().astype(np.float64) - theta0)
    assert np.median(moved[sure]) > 0.5 * lr


def test_block_features_of_hand_built_tensor(df):
    """The library's features of the hand-built tensor whose 16 values per block are
    worked out by hand in the oracle's pins (a ragged block of 2 functions included)."""
    from test_oracle_mlp import hand_features, hand_tensor
    B, _ = hand_tensor()
    ctx = df.Context(2, 130, 4)
    Bg = torch.from_numpy(B).cuda()
    ctx.setup(Bg)
    F = df.block_features(ctx, 4, 1e-10, 1e-4, 1e-8, 5).cpu().numpy()
    assert np.allclose(F, hand_features(), rtol=0, atol=2e-7)


def test_mlp_training_fits_a_small_set(df):
    rng = np.random.default_rng(6)
    X = rng.standard_normal((64, 16)).astype(np.float32)
    y = rng.integers(0, 8, size=64)
    from paper_2601_08077_gb300 import predictor
    p = predictor.SlicePredictor(seed=1)
    hist = p.fit(torch.from_numpy(X).cuda(), torch.from_numpy(y.astype(np.int32)).cuda(), steps=800, lr=1e-2)
    assert hist[-1] < 0.2 * hist[0]
    pred = p.mlp.forward(torch.from_numpy(X).cuda()).cpu().numpy().argmax(1)
    assert np.mean(pred == y) > 0.9


@pytest.fixture(scope="module")
def small_ctx(df):
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    ctx = df.Context(mol.nao, mol.naux, C.shape[1])
    Bg = torch.from_numpy(B).cuda()
    ctx.setup(Bg)
    return ctx, Bg, B, C


def test_block_features_match_oracle(df, small_ctx):
    ctx, Bg, B, C = small_ctx
    F = df.block_features(ctx, C.shape[1], 1e-10, 3e-4, 2e-9, 5).cpu().numpy()
    rows = B.reshape(-1, B.shape[2])
    eB, _ = O.split_rows(rows, 1)
    F_ref = M.block_features(B, eB, C.shape[1], 1e-10, 3e-4, 2e-9, 5)
    assert np.max(np.abs(F - F_ref)) < 1e-5


def test_block_errors_against_oracle(df, small_ctx):
    ctx, Bg, B, C = small_ctx
    err, kmax = df.block_errors(ctx, torch.from_numpy(C).cuda())
    K = O.exchange(B, C)
    assert abs(kmax - np.max(np.abs(K))) <= 1e-13 * kmax
    X = O.exchange_X(B, C)
    nao = B.shape[1]
    for s in (3, 5):
        _, _, parts = O.emulated_exchange(B, C, s, return_parts=True)
        for b, Kb in enumerate(parts):
            Xb = X[b * 128:(b + 1) * 128].transpose(1, 0, 2).reshape(nao, -1)
            ref = np.max(np.abs(Kb - Xb @ Xb.T))
            assert abs(err[b, s - 1] - ref) <= 1e-14 * kmax + 1e-3 * ref
    assert np.all(err[:, 7] <= 1e-13 * kmax)
    assert np.all(err[:, 2] > err[:, 5])


def _constant_network(df, cls, logit=10.0):
    """A network whose output is class `cls` (count cls + 1) with confidence ~1 for any input."""
    theta = np.zeros(M.N_PARAMS, dtype=np.float32)
    theta[M.N_PARAMS - 8 + cls] = logit       # b3
    return df.MLP(theta)


def _at_level_2(ctx):
    """Drive the context's controller to Table 1 level 2 (count 5): dE_rel = 1e-10."""
    ctx.adaptive_reset()
    ctx.adaptive_next(100.0)
    assert ctx.adaptive_next(100.0 + 1e-8) == (2, 5)


def test_adaptive_mode_runs_the_controllers_count(df, small_ctx):
    ctx, Bg, B, C = small_ctx
    Cg = torch.from_numpy(C).cuda()
    ctx.adaptive_reset()
    K, st = ctx.build_K(Cg, df.ADAPTIVE)
    assert st.level == 4 and list(st.slices[:st.nblk]) == [3] * st.nblk and st.slice_pairs == 6 * st.nblk
    assert torch.equal(K, ctx.build_K(Cg, 3)[0])
    _at_level_2(ctx)
    K, st = ctx.build_K(Cg, df.ADAPTIVE)
    assert st.level == 2 and list(st.slices[:st.nblk]) == [5] * st.nblk
    assert np.array_equal(K.cpu().numpy(), O.emulated_exchange(B, C, 5))


def test_learned_mode_needs_a_network(df, small_ctx):
    ctx, Bg, B, C = small_ctx
    ctx.set_predictor(None)
    _at_level_2(ctx)
    with pytest.raises(df.DFError):
        ctx.build_K(torch.from_numpy(C).cuda(), df.LEARNED)


def test_learned_mode_low_confidence_falls_back_to_the_rule(df, small_ctx):
    """All-zero parameters give probability 1/8 per count, below the 0.6 threshold:
    every block takes the level's count, nothing is recomputed."""
    ctx, Bg, B, C = small_ctx
    net = df.MLP(np.zeros(M.N_PARAMS, dtype=np.float32))
    ctx.set_predictor(net, 0.6)
    _at_level_2(ctx)
    K, st = ctx.build_K(torch.from_numpy(C).cuda(), df.LEARNED)
    assert st.low_confidence == st.nblk and st.recomputed == 0 and st.level == 2
    assert np.array_equal(K.cpu().numpy(), O.emulated_exchange(B, C, 5))
    ctx.set_predictor(None)


def test_learned_mode_check_recomputes_the_blocks_that_miss(df):
    """Host-side input choice forces misses: the last auxiliary block of the 20-atom molecule
    is scaled by 2^-40 and the network asks 4 slices everywhere at level 2 (count 5).  The
    FP64-free bound check keeps 4 slices only where the bound allows it (the scaled block,
    whose bound is ~2^-80 of the others), raises the other two blocks to 5 and recomputes
    them; K is then exactly the oracle's emulation with counts [5, 5, 4] and within the
    1e-10 target of the oracle's exact K."""
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    B = B.copy()
    B[256:] *= 2.0 ** -40
    ctx = df.Context(mol.nao, mol.naux, C.shape[1])
    Bg = torch.from_numpy(B).cuda()
    ctx.setup(Bg)
    net = _constant_network(df, 3)
    ctx.set_predictor(net, 0.6)
    _at_level_2(ctx)
    K, st = ctx.build_K(torch.from_numpy(C).cuda(), df.LEARNED)
    assert st.recomputed == 2 and list(st.slices[:3]) == [5, 5, 4] and st.low_confidence == 0
    assert st.bound_ratio <= 1.0 + 1e-12 and st.slice_pairs == 15 + 15 + 10
    got = K.cpu().numpy()
    assert np.array_equal(got, O.emulated_exchange(B, C, [5, 5, 4]))
    K_ref = O.exchange(B, C)
    assert np.max(np.abs(got - K_ref)) <= 1e-10 * np.max(np.abs(K_ref))
    # a network asking 1 slice everywhere: the scaled block's bound is still ~1e-15 of the
    # total, so only the other two are raised
    net1 = _constant_network(df, 0)
    ctx.set_predictor(net1, 0.6)
    K1, st1 = ctx.build_K(torch.from_numpy(C).cuda(), df.LEARNED)
    assert st1.recomputed == 2 and list(st1.slices[:3]) == [5, 5, 1]
    assert np.array_equal(K1.cpu().numpy(), O.emulated_exchange(B, C, [5, 5, 1]))
    # on the unscaled molecule every block is raised
    ctx0 = df.Context(mol.nao, mol.naux, C.shape[1])
    B0 = torch.from_numpy(inputs.make_inputs(inputs.SMALL)[1]).cuda()
    ctx0.setup(B0)
    ctx0.set_predictor(net1, 0.6)
    _at_level_2(ctx0)
    K0, st0 = ctx0.build_K(torch.from_numpy(C).cuda(), df.LEARNED)
    assert st0.recomputed == 3 and list(st0.slices[:3]) == [5, 5, 5]
    assert np.array_equal(K0.cpu().numpy(), O.emulated_exchange(B0.cpu().numpy(), C, 5))


def test_learned_mode_keeps_counts_that_pass(df):
    """A hand-set network that asks one slice more than the level on blocks near the
    largest scale and one slice less on blocks more than 20 binades below it (feature 13):
    the check passes without a recompute and K is the oracle's emulation at those counts
    (level 3, count 4: the counts stay <= 5, where the recombination keeps every bit)."""
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    B = B.copy()
    B[256:] *= 2.0 ** -40
    ctx = df.Context(mol.nao, mol.naux, C.shape[1])
    Bg = torch.from_numpy(B).cuda()
    ctx.setup(Bg)
    d = {name: np.zeros(shape) for name, shape in M.SHAPES}
    d["W1"][0, 13] = -32.0            # h1_0 = binades below the largest block
    d["W2"][0, 0], d["b2"][0] = 1.0, -20.0
    d["W3"][2, 0] = 1.0               # class 2 (3 slices) grows with the binades beyond 20
    d["b3"][4] = 5.0                  # class 4 (5 slices) otherwise
    net = df.MLP(M.pack(d).astype(np.float32))
    ctx.set_predictor(net, 0.6)
    ctx.adaptive_reset()
    ctx.adaptive_next(100.0)
    assert ctx.adaptive_next(100.0 + 1e-5) == (3, 4)      # dE_rel = 1e-7: level 3
    K, st = ctx.build_K(torch.from_numpy(C).cuda(), df.LEARNED)
    assert list(st.slices[:3]) == [5, 5, 3] and st.recomputed == 0 and st.low_confidence == 0
    assert st.bound_ratio < 1.0 and st.level == 3
    assert np.array_equal(K.cpu().numpy(), O.emulated_exchange(B, C, [5, 5, 3]))


def test_block_errors_of_an_ordered_setup_against_oracle(df, small_ctx):
    """With the auxiliary functions in magnitude order, block b of the errors is block b of
    the permuted tensor: emulated and FP64 K_b both over the permuted block's functions."""
    ctx0, Bg, B, C = small_ctx
    perm = np.argsort(-np.abs(B).reshape(B.shape[0], -1).max(1))
    ctx = df.Context(B.shape[1], B.shape[0], C.shape[1])
    ctx.setup(Bg, perm=perm)
    err, kmax = df.block_errors(ctx, torch.from_numpy(C).cuda())
    Bp = B[perm]
    X = O.exchange_X(Bp, C)
    nao = B.shape[1]
    for s in (3, 5):
        _, _, parts = O.emulated_exchange(Bp, C, s, return_parts=True)
        for b, Kb in enumerate(parts):
            Xb = X[b * 128:(b + 1) * 128].transpose(1, 0, 2).reshape(nao, -1)
            ref = np.max(np.abs(Kb - Xb @ Xb.T))
            assert abs(err[b, s - 1] - ref) <= 1e-14 * kmax + 1e-3 * ref
    assert np.all(err[:, 2] > 100 * err[:, 4])


def test_ordered_setup_matches_oracle_on_permuted_tensor(df, small_ctx):
    ctx0, Bg, B, C = small_ctx
    perm = np.argsort(-np.abs(B).reshape(B.shape[0], -1).max(1))
    ctx = df.Context(B.shape[1], B.shape[0], C.shape[1])
    ctx.setup(Bg, perm=perm)
    Cg = torch.from_numpy(C).cuda()
    K = ctx.build_K(Cg, 5)[0].cpu().numpy()
    assert np.array_equal(K, O.emulated_exchange(B[perm], C, 5))
    D = torch.from_numpy(inputs.density(C)).cuda()
    J = ctx.build_J(D)[0]
    assert torch.equal(J, ctx0.build_J(D)[0])


def test_learned_counts_state_the_gain_on_a_held_out_molecule(df):
    """The learned part's gain, stated.  Train on twelve molecules of 20-40 atoms (labels: per
    level, the fewest slice pairs whose summed block errors stay within the rule's), then
    run the library's learned mode on a held-out 36-atom molecule at every level.

    What holds: the check keeps the learned build's error bound within the rule's, and the
    learned K is as accurate as the rule's (against FP64).  What it gains: on these
    molecules the 128-function blocks' errors at a given count stay within ~30x of each
    other, so no trade of slices between blocks pays (one slice changes a block's error by
    16-256x, and raising a block costs s + 1 pairs where lowering one saves s): the labels
    themselves save under 5 % of the rule's slice pairs, and the network saves no more."""
    from paper_2601_08077_gb300 import predictor
    train, keep = [], []
    for atoms, seed in [(20, 21), (26, 22), (30, 23), (34, 24), (24, 25), (38, 26), (22, 27), (28, 28),
                        (32, 29), (36, 30), (40, 33), (21, 34)]:
        mol = inputs.molecule(atoms, seed)
        B = inputs.df_tensor_device(mol)
        ctx = df.Context(mol.nao, mol.naux, atoms)
        ctx.setup(B, perm=predictor.magnitude_order(B))
        C = torch.from_numpy(inputs.orbitals(mol.nao, atoms, seed + 1)).cuda()
        F, y, _, _ = predictor.molecule_dataset(ctx, C)
        train.append((F, y))
        keep.append((ctx, B))
    F = torch.cat([t[0] for t in train])
    y = torch.cat([t[1] for t in train])
    p = predictor.SlicePredictor(seed=0)
    hist = p.fit(F, y, steps=2500, lr=3e-3)
    assert hist[-1] < hist[0]
    mol = inputs.molecule(36, 31)
    B = inputs.df_tensor_device(mol)
    ctx = df.Context(mol.nao, mol.naux, 36)
    ctx.setup(B, perm=predictor.magnitude_order(B))
    C = torch.from_numpy(inputs.orbitals(mol.nao, 36, 32)).cuda()
    err, kmax = df.block_errors(ctx, C)
    K64 = ctx.build_K(C, 0)[0].clone()
    p.attach(ctx)
    work = {"rule": 0, "labels": 0, "learned": 0}
    recomputed = 0
    for level, dE in ((4, 1e-5), (3, 1e-7), (2, 1e-10), (1, 1e-12)):
        ctx.adaptive_reset()
        ctx.adaptive_next(100.0)
        assert ctx.adaptive_next(100.0 * (1.0 + dE))[0] == level
        s_rule = predictor.LEVELS[level][1]
        K_rule, st_rule = ctx.build_K(C, df.ADAPTIVE)
        K_l, st_l = ctx.build_K(C, df.LEARNED)
        assert st_l.level == level and st_l.bound_ratio <= 1.0 + 1e-12
        e_rule = float((K_rule - K64).abs().max())
        e_l = float((K_l - K64).abs().max())
        assert e_l <= 2.0 * e_rule + 1e-15 * kmax
        work["rule"] += st_rule.slice_pairs
        work["learned"] += st_l.slice_pairs
        work["labels"] += sum(predictor.pairs(int(s)) for s in predictor.labels_at_rule_accuracy(err, s_rule))
        recomputed += st_l.recomputed
    gain_labels = 1.0 - work["labels"] / work["rule"]
    gain_learned = 1.0 - work["learned"] / work["rule"]
    print("slice pairs: rule %(rule)d, labels %(labels)d, learned %(learned)d" % work,
          "recomputed %d; gain labels %.3f learned %.3f" % (recomputed, gain_labels, gain_learned))
    assert 0.0 <= gain_labels < 0.05
    assert -0.10 < gain_learned < 0.05      # no gain; at most the cost of a few misplaced counts
