"""CPU oracle of the learned slice predictor (TEST INFRASTRUCTURE ONLY).

Plain NumPy FP64 restatement of the 16 -> 64 -> 64 -> 8 ReLU MLP with a
softmax over the slice counts 1..8, its mean cross-entropy and its gradients
by backpropagation, of the label rules (the least slice count whose per-block
K error meets the block's share of a tolerance; the per-block counts of fewest
slice pairs whose summed block errors stay within the rule's) and of the block
features.
The predictor is not in the paper; it extends the paper's closing suggestion
(Section 5) of tying the emulation level to the change of the density matrix,
with the per-block error budget read as an additive split of the tolerance.
Training uses Adam (Kingma and Ba, 2015: moments with decay 0.9 / 0.999, bias
correction by 1 - beta^t, eps 1e-8), restated in ``adam_step``.

Pins (tests/test_oracle_mlp.py): backpropagation against finite
differences; the forward pass of a hand-set network whose logits are worked
out by hand (a missing ReLU or a transposed weight fails it); Adam's closed
forms (first step lr sign(g), constant gradient, zero gradient); the block
features of a hand-built tensor whose 16 values are worked out by hand.

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


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns (theta', m', v').

    m' = beta1 m + (1 - beta1) g, v' = beta2 v + (1 - beta2) g^2,
    theta' = theta - lr (m' / (1 - beta1^t)) / (sqrt(v' / (1 - beta2^t)) + eps).
    """
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return np.asarray(theta, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v


def labels(err, kmax, tau, nblk):
    """Least s (1..8) with max|K_b(s) - K_b(FP64)| <= tau max|K| / nblk; 8 if none."""
    budget = tau * kmax / nblk
    out = np.full(err.shape[0], 8, dtype=np.int64)
    for b in range(err.shape[0]):
        ok = np.nonzero(err[b] <= budget)[0]
        if len(ok):
            out[b] = ok[0] + 1
    return out


def labels_at_rule_accuracy(err, s_rule):
    """Per-block slice counts (1..8) with the fewest slice pairs sum_b s_b (s_b + 1) / 2
    whose summed block errors stay within the rule's: sum_b err[b, s_b - 1] <=
    sum_b err[b, s_rule - 1] (err[b, s - 1] = max|K_b(s) - K_b(FP64)|).  The
    definition, by enumerating every assignment (tiny nblk only); ties go to the
    smaller error sum, then to the lexicographically larger counts."""
    import itertools
    err = np.asarray(err, dtype=np.float64)
    nblk = err.shape[0]
    budget = float(np.sum(err[:, s_rule - 1]))
    best = None
    for combo in itertools.product(range(1, 9), repeat=nblk):
        e = float(sum(err[b, combo[b] - 1] for b in range(nblk)))
        if e > budget:
            continue
        key = (sum(s * (s + 1) // 2 for s in combo), e, tuple(-s for s in combo))
        if best is None or key < best[0]:
            best = (key, combo)
    return np.array(best[1], dtype=np.int64)


def block_features(B, eB, nocc, tau, dD, dE, s_rule, block=128):
    """The 16 input features of every auxiliary block b (rows P in the block).

    With Bb the block's slice of B, eB the per-(P, mu) row exponents of the
    split (a zero row counts with exponent 0), rows = all (P, mu) rows of the
    block, Emax / Emin their largest / smallest exponent, ss_b = sum Bb^2 and
    max_b = max|Bb|:

      0  log2(max_b) / 32                  8  log2(nao) / 12
      1  log2(sqrt(ss_b)) / 32             9  log2(nocc) / 10
      2  mean of eB over rows / 32         10 log2(ss_b / sum_b' ss_b') / 32
      3  (Emax - Emin) / 32                11 fraction of rows with eB < Emax - 20
      4  log10(tau) / 16                   12 s_rule / 8
      5  log10(dD + 1e-30) / 16            13 (log2(max_b) - log2(max_b' max_b')) / 32
      6  b / nblk                          14 log10(dE + 1e-30) / 16
      7  log2(number of P in the block) / 8  15 1 (bias input)

    A tiny 1e-300 is added inside every log2 of a norm, so an all-zero block
    gives finite features.
    """
    naux, nao, _ = B.shape
    nblk = (naux + block - 1) // block
    tiny = 1e-300
    maxes, sums = [], []
    for b in range(nblk):
        Bb = B[b * block:(b + 1) * block]
        maxes.append(float(np.abs(Bb).max()))
        sums.append(float(np.sum(Bb * Bb)))
    gmax, gss = max(maxes), sum(sums)
    F = np.zeros((nblk, 16))
    for b in range(nblk):
        p0, p1 = b * block, min((b + 1) * block, naux)
        e = np.asarray(eB[p0 * nao:p1 * nao], dtype=np.float64)
        emax, emin = e.max(), e.min()
        F[b, 0] = np.log2(maxes[b] + tiny) / 32
        F[b, 1] = 0.5 * np.log2(sums[b] + tiny) / 32
        F[b, 2] = e.mean() / 32
        F[b, 3] = (emax - emin) / 32
        F[b, 4] = np.log10(tau) / 16
        F[b, 5] = np.log10(dD + 1e-30) / 16
        F[b, 6] = b / nblk
        F[b, 7] = np.log2(p1 - p0) / 8
        F[b, 8] = np.log2(nao) / 12
        F[b, 9] = np.log2(nocc) / 10
        F[b, 10] = np.log2(sums[b] / max(gss, tiny) + tiny) / 32
        F[b, 11] = np.count_nonzero(e < emax - 20) / len(e)
        F[b, 12] = s_rule / 8
        F[b, 13] = (np.log2(maxes[b] + tiny) - np.log2(gmax + tiny)) / 32
        F[b, 14] = np.log10(dE + 1e-30) / 16
        F[b, 15] = 1.0
    return F
