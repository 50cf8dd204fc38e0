"""Pins of the predictor oracle: backpropagation against finite differences, softmax, labels,
a hand-set network, Adam's closed forms and the features of a hand-built tensor."""
import math

import numpy as np

from oracle import df_oracle as O
from oracle import mlp_oracle as M


def test_param_count_and_layout():
    assert M.N_PARAMS == 16 * 64 + 64 + 64 * 64 + 64 + 8 * 64 + 8
    th = np.arange(M.N_PARAMS, dtype=float)
    assert np.array_equal(M.pack(M.unpack(th)), th)


def test_softmax_rows_sum_to_one_and_uniform_at_zero():
    X = np.random.default_rng(0).standard_normal((5, 16))
    probs, _ = M.forward(np.zeros(M.N_PARAMS), X)
    assert np.allclose(probs, 1.0 / 8)
    probs, _ = M.forward(M.init_params(3), X)
    assert np.allclose(probs.sum(1), 1.0)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    th = M.init_params(2) + 0.01 * rng.standard_normal(M.N_PARAMS)
    X = rng.standard_normal((7, 16))
    y = rng.integers(0, 8, size=7)
    g = M.gradients(th, X, y)
    idx = rng.choice(M.N_PARAMS, size=60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(M.N_PARAMS)
        e[i] = h
        fd = (M.loss(th + e, X, y) - M.loss(th - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd)


def test_labels_pick_least_slice_count_within_budget():
    err = np.array([[1e-1, 1e-3, 1e-6, 1e-9, 1e-12, 1e-14, 1e-15, 1e-16],
                    [1e-2, 1e-2, 1e-2, 1e-2, 1e-2, 1e-2, 1e-2, 1e-2]])
    lab = M.labels(err, kmax=2.0, tau=1e-10, nblk=2)     # budget 1e-10
    assert list(lab) == [5, 8]


# --- the forward pass of a hand-set network --------------------------------------

def hand_network():
    """Weights set by hand (everything else zero):
    h1_0 = relu(x0 + 2 x1 - 1), h1_1 = relu(-x0 + 1/2),
    h2_0 = relu(h1_0 - 3 h1_1 + 1/4), h2_1 = relu(2 h1_1),
    z_0 = h2_0, z_1 = h2_1, z_2 = h2_0 - h2_1 + 1, z_3..7 = 0."""
    d = {name: np.zeros(shape) for name, shape in M.SHAPES}
    d["W1"][0, 0], d["W1"][0, 1], d["b1"][0] = 1.0, 2.0, -1.0
    d["W1"][1, 0], d["b1"][1] = -1.0, 0.5
    d["W2"][0, 0], d["W2"][0, 1], d["b2"][0] = 1.0, -3.0, 0.25
    d["W2"][1, 1] = 2.0
    d["W3"][0, 0], d["W3"][1, 1], d["W3"][2, 0], d["W3"][2, 1], d["b3"][2] = 1.0, 1.0, 1.0, -1.0, 1.0
    return M.pack(d)


def softmax_of(z):
    e = [math.exp(v - max(z)) for v in z]
    return [v / sum(e) for v in e]


def test_forward_of_hand_set_network():
    X = np.zeros((2, 16))
    X[0, :2] = (1.0, 0.5)     # h1 = (1, 0) [relu cuts -1/2], h2 = (5/4, 0)
    X[1, :2] = (-1.0, 0.25)   # h1 = (0, 3/2) [relu cuts -3/2], h2 = (0, 3) [relu cuts -17/4]
    z_by_hand = [[1.25, 0.0, 2.25, 0, 0, 0, 0, 0], [0.0, 3.0, -2.0, 0, 0, 0, 0, 0]]
    probs, (a1, h1, a2, h2) = M.forward(hand_network(), X)
    assert np.allclose(a1[:, :2], [[1.0, -0.5], [-1.5, 1.5]], rtol=0, atol=1e-15)
    assert np.allclose(h2[:, :2], [[1.25, 0.0], [0.0, 3.0]], rtol=0, atol=1e-15)
    for r in range(2):
        assert np.allclose(probs[r], softmax_of(z_by_hand[r]), rtol=1e-14, atol=0)
    y = np.array([2, 1])
    want = -0.5 * (math.log(softmax_of(z_by_hand[0])[2]) + math.log(softmax_of(z_by_hand[1])[1]))
    assert abs(M.loss(hand_network(), X, y) - want) < 1e-14


# --- Adam ---------------------------------------------------------------------------

def test_adam_first_step_moves_by_lr_times_sign():
    """Zero moments: m^ = g and v^ = g^2 after one step, so the update is lr g / (|g| + eps)."""
    g = np.array([3.0, -0.5, 1e-3, 0.0, -2e-6])
    th0 = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    th1, m, v = M.adam_step(th0, g, np.zeros(5), np.zeros(5), 1, 0.01)
    assert np.allclose(th1, th0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-16)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_takes_equal_steps():
    g = np.array([0.7, -4.0])
    th, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    for t in range(1, 6):
        th, m, v = M.adam_step(th, g, m, v, t, 1e-3)
    assert np.allclose(th, -5 * 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_adam_reversed_gradient_second_step():
    """g then -g: m2 = -(1-b1)^2 g, m^2 = -(1-b1)/(1+b1) g = -g/19; v^2 = g^2: the second
    update is +lr sign(g)/19."""
    g = np.array([2.0, -0.25])
    th1, m, v = M.adam_step(np.zeros(2), g, np.zeros(2), np.zeros(2), 1, 0.1)
    th2, m, v = M.adam_step(th1, -g, m, v, 2, 0.1)
    assert np.allclose(th2 - th1, 0.1 * np.sign(g) / 19 * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_adam_zero_gradient_keeps_parameters():
    th, m, v = M.adam_step(np.array([1.5]), np.array([0.0]), np.array([0.0]), np.array([0.0]), 1, 0.5)
    assert th[0] == 1.5


# --- block features of a hand-built tensor ---------------------------------------------

def hand_tensor():
    """naux 130 (one full 128-function block and a ragged block of 2), nao 2.
    Block 0: B_P = [[1, 0], [0, 0]], except B_5 = [[4, 0], [0, 2^-30]] and
    B_6 = [[1, 0], [0, 2^-18]].
    Block 1: B_P = [[2^-10, 2^-10], [2^-10, 0]].
    Row exponents (smallest e with max|row| < 127/128 2^e; zero rows 0):
    rows (P, 0) 1 and (P, 1) 0 in block 0, except (5, 0) 3, (5, 1) -29 and
    (6, 1) -17 (exactly Emax - 20: not a small row); every row of block 1 -9."""
    B = np.zeros((130, 2, 2))
    B[:128, 0, 0] = 1.0
    B[5, 0, 0], B[5, 1, 1] = 4.0, 2.0 ** -30
    B[6, 1, 1] = 2.0 ** -18
    B[128:] = [[2.0 ** -10, 2.0 ** -10], [2.0 ** -10, 0.0]]
    eB = np.zeros(260, dtype=np.int64)
    eB[0:256:2] = 1
    eB[10], eB[11] = 3, -29
    eB[13] = -17
    eB[256:] = -9
    return B, eB


def hand_features():
    ss0 = 127.0 + 16.0 + 2.0 ** -60 + 2.0 ** -36
    ss1 = 2 * 3 * 2.0 ** -20
    common = {4: -10 / 16, 5: math.log10(1e-4 + 1e-30) / 16, 8: 1 / 12, 9: 2 / 10, 12: 5 / 8, 14: -8 / 16, 15: 1.0}
    f0 = dict(common)
    f0.update({0: 2 / 32, 1: 0.5 * math.log2(ss0) / 32, 2: (127 * 1 + 3 - 29 - 17) / 256 / 32, 3: 32 / 32, 6: 0.0,
               7: 7 / 8, 10: math.log2(ss0 / (ss0 + ss1)) / 32, 11: 1 / 256, 13: 0.0})
    f1 = dict(common)
    f1.update({0: -10 / 32, 1: 0.5 * math.log2(ss1) / 32, 2: -9 / 32, 3: 0.0, 6: 0.5, 7: 1 / 8,
               10: math.log2(ss1 / (ss0 + ss1)) / 32, 11: 0.0, 13: -12 / 32})
    return np.array([[f0[k] for k in range(16)], [f1[k] for k in range(16)]])


def test_block_features_of_hand_built_tensor():
    B, eB = hand_tensor()
    assert np.array_equal(O.row_exponents(B.reshape(-1, 2)), eB)
    F = M.block_features(B, eB, nocc=4, tau=1e-10, dD=1e-4, dE=1e-8, s_rule=5)
    assert F.shape == (2, 16)
    assert np.allclose(F, hand_features(), rtol=0, atol=1e-15)


def test_labels_at_rule_accuracy_hand_table():
    """Three blocks, errors 256x per slice: block 0 dominates (scale 1), blocks 1 and 2 are
    10^-4 of it.  At the rule's 4 slices (10 pairs each, 30 in all) the budget is
    (1 + 2e-4) 256^-4; raising block 0 to 5 frees 255/256 of its share, which pays for
    lowering both small blocks to 3 (each adds 255e-4 256^-4): 15 + 6 + 6 = 27 pairs."""
    err = np.array([[1.0 * 256.0 ** -s for s in range(1, 9)],
                    [1e-4 * 256.0 ** -s for s in range(1, 9)],
                    [1e-4 * 256.0 ** -s for s in range(1, 9)]])
    assert list(M.labels_at_rule_accuracy(err, 4)) == [5, 3, 3]
    # equal blocks: nothing to trade, the rule's own counts
    eq = np.array([[256.0 ** -s for s in range(1, 9)]] * 3)
    assert list(M.labels_at_rule_accuracy(eq, 4)) == [4, 4, 4]
