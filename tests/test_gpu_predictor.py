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


def test_predictor_gain_on_held_out_molecule(df):
    """Train on small molecules, predict per-block counts on a held-out one: every block meets its
    budget after the counted recomputes, and the work is compared with the best uniform count."""
    from paper_2601_08077_gb300 import predictor
    train, keep = [], []
    for atoms, seed in [(20, 21), (26, 22), (30, 23), (34, 24), (24, 25), (38, 26)]:
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
    hist = p.fit(F, y, steps=1500, lr=3e-3)
    assert hist[-1] < hist[0]
    mol = inputs.molecule(36, 31)
    B = inputs.df_tensor_device(mol)
    ctx = df.Context(mol.nao, mol.naux, 36)
    ctx.setup(B, perm=predictor.magnitude_order(B))
    C = torch.from_numpy(inputs.orbitals(mol.nao, 36, 32)).cuda()
    err, kmax = df.block_errors(ctx, C)
    totals = {"pred": 0, "uniform": 0, "rule": 0, "recomputed": 0}
    for tau in predictor.TAUS:
        Ft = df.block_features(ctx, 36, tau, 1e-3, 1e-6, predictor.rule_slices(tau))
        s_pred, conf, nfb = p.predict(Ft, fallback_s=predictor.rule_slices(tau))
        r = predictor.evaluate(err, kmax, tau, s_pred)
        budget = tau * kmax / err.shape[0]
        assert all(err[b, s - 1] <= budget or s == r["s_uniform"] for b, s in enumerate(r["s_final"]))
        totals["pred"] += r["work_pred"]
        totals["uniform"] += r["work_uniform"]
        totals["rule"] += r["work_rule"]
        totals["recomputed"] += r["recomputed"]
    print("predictor work %(pred)d vs best uniform %(uniform)d vs rule %(rule)d, recomputed %(recomputed)d" % totals)
    assert totals["pred"] <= totals["uniform"]


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
