"""Pins of the predictor oracle: backpropagation against finite differences, softmax, labels."""
import numpy as np

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
