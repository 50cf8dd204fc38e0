"""CPU oracle of the learned slice predictor (TEST INFRASTRUCTURE ONLY).

Plain NumPy FP64 restatement of the 16 -> 64 -> 64 -> 8 ReLU MLP with a
softmax over the slice counts 1..8, its mean cross-entropy and its gradients
by backpropagation, of the label rule (the least slice count whose per-block
K error meets the block's share of the tolerance) and of the block features.
The predictor is not in the paper; it extends the paper's closing suggestion
(Section 5) of tying the emulation level to the change of the density matrix,
with the per-block error budget read as an additive split of the tolerance.

Parameter layout (as in the CUDA library): W1[64][16], b1[64], W2[64][64],
b2[64], W3[8][64], b3[8].
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 16, 64, 8
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_OUT, N_H)),
          ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([d[name].ravel() for name, _ in SHAPES])


def init_params(seed):
    """He-normal weights, zero biases (the seeded draw both sides start from)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SHAPES:
        d[name] = rng.standard_normal(shape) * np.sqrt(2.0 / shape[1]) if name.startswith("W") else np.zeros(shape)
    return pack(d)


def forward(theta, X):
    p = unpack(theta)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"].T + p["b3"]
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    probs = e / e.sum(axis=1, keepdims=True)
    return probs, (a1, h1, a2, h2)


def loss(theta, X, y):
    probs, _ = forward(theta, X)
    return float(-np.mean(np.log(probs[np.arange(len(y)), y])))


def gradients(theta, X, y):
    """d loss / d theta of the mean cross-entropy, by backpropagation."""
    p = unpack(theta)
    probs, (a1, h1, a2, h2) = forward(theta, X)
    n = len(y)
    dz = probs.copy()
    dz[np.arange(n), y] -= 1.0
    dz /= n
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    dh2 = (dz @ p["W3"]) * (a2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ p["W2"]) * (a1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(0)
    return pack(g)


def labels(err, kmax, tau, nblk):
    """Least s (1..8) with max|K_b(s) - K_b(FP64)| <= tau max|K| / nblk; 8 if none."""
    budget = tau * kmax / nblk
    out = np.full(err.shape[0], 8, dtype=np.int64)
    for b in range(err.shape[0]):
        ok = np.nonzero(err[b] <= budget)[0]
        if len(ok):
            out[b] = ok[0] + 1
    return out


def block_features(B, eB, nocc, tau, dD, dE, s_rule, block=128):
    """The 16 features of every block (same definitions and scalings as the library)."""
    naux, nao, _ = B.shape
    nblk = (naux + block - 1) // block
    st = []
    for b in range(nblk):
        Bb = B[b * block:(b + 1) * block]
        e = eB[b * block * nao:(b * block + Bb.shape[0]) * nao].astype(np.float64)
        st.append((np.abs(Bb).max(), float((Bb * Bb).sum()), e.sum(), float(len(e)), e.min(), e.max(),
                   float(np.sum(e < e.max() - 20))))
    st = np.array(st)
    gmax, gss = st[:, 0].max(), st[:, 1].sum()
    F = np.zeros((nblk, 16))
    tiny = 1e-300
    for b in range(nblk):
        mx, ss, es, cnt, emin, emax, small = st[b]
        nP = min(block, naux - b * block)
        F[b] = [np.log2(mx + tiny) / 32, 0.5 * np.log2(ss + tiny) / 32, es / max(cnt, 1) / 32, (emax - emin) / 32,
                np.log10(tau) / 16, np.log10(dD + 1e-30) / 16, b / nblk, np.log2(nP) / 8, np.log2(nao) / 12,
                np.log2(nocc) / 10, np.log2(ss / max(gss, tiny) + tiny) / 32, small / max(cnt, 1), s_rule / 8,
                (np.log2(mx + tiny) - np.log2(gmax + tiny)) / 32, np.log10(dE + 1e-30) / 16, 1.0]
    return F
