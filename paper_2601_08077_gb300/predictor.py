"""Learned per-block slice counts for the exchange build.

The network (16 block features -> 64 -> 64 -> 8 slice counts) runs and trains
on the device through libdf's own kernels.  Its labels come from the method
itself: for every 128-function auxiliary block, the least slice count whose
K error against the native FP64 build stays within the block's share of the
tolerance (tau max|K| / nblk, an additive split that bounds the total).  At
run time a prediction below the confidence threshold falls back to the slice
count of the paper's rule (Table 1) for the same tolerance, and a block that
misses its budget is recomputed at that count and counted.
"""
from __future__ import annotations

import numpy as np
import torch

from . import df

# Table 1's printed accuracies (levels 4..1) and the 1e-10 target of the K error
TAUS = (1.2e-7, 4.7e-10, 1e-10, 1.8e-12, 7.1e-15)


def rule_slices(tau: float) -> int:
    """Slice count of the Table 1 level whose printed accuracy is at least as tight as tau."""
    for acc, s in ((1.2e-7, 3), (4.7e-10, 4), (1.8e-12, 5), (7.1e-15, 6)):
        if acc <= tau:
            return s
    return 8


def pairs(s):
    return s * (s + 1) // 2


def labels_from_errors(err: np.ndarray, kmax: float, tau: float) -> np.ndarray:
    """Least s in 1..8 with err[b, s-1] <= tau kmax / nblk (8 if none)."""
    nblk = err.shape[0]
    budget = tau * kmax / nblk
    ok = err <= budget
    lab = np.where(ok.any(axis=1), ok.argmax(axis=1) + 1, 8)
    return lab.astype(np.int64)


def init_params(seed: int) -> np.ndarray:
    """He-normal weights and zero biases, in the library's parameter layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for rows, cols in ((64, 16), (64, 0), (64, 64), (64, 0), (8, 64), (8, 0)):
        if cols:
            parts.append(rng.standard_normal((rows, cols)) * np.sqrt(2.0 / cols))
        else:
            parts.append(np.zeros(rows))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def magnitude_order(B: torch.Tensor) -> np.ndarray:
    """Auxiliary functions by decreasing max|B_P| (for df_setup_ordered): blocks of similar scale."""
    return torch.argsort(B.abs().amax(dim=(1, 2)), descending=True).cpu().numpy()


def molecule_dataset(ctx, C, taus=TAUS, seed=0):
    """Features and labels of every block of one molecule at every tolerance.

    The density-change and energy-change features are drawn log-uniformly over
    the range an SCF-like sequence visits (the labels do not depend on them).
    """
    rng = np.random.default_rng(seed)
    err, kmax = df.block_errors(ctx, C)
    Fs, ys = [], []
    for tau in taus:
        dD = 10.0 ** rng.uniform(-14, 0)
        dE = 10.0 ** rng.uniform(-16, -2)
        Fs.append(df.block_features(ctx, C.shape[1], tau, dD, dE, rule_slices(tau)))
        ys.append(torch.from_numpy(labels_from_errors(err, kmax, tau) - 1).to(torch.int32).cuda())
    return torch.cat(Fs), torch.cat(ys), err, kmax


class SlicePredictor:
    def __init__(self, seed: int = 0):
        self.mlp = df.MLP(init_params(seed))

    def fit(self, F: torch.Tensor, y: torch.Tensor, steps: int = 2000, lr: float = 3e-3, batch: int = 0,
            seed: int = 0):
        """Adam on the mean cross-entropy; full batch unless `batch` > 0.  Returns the loss history."""
        g = torch.Generator(device="cpu").manual_seed(seed)
        hist = []
        n = F.shape[0]
        for it in range(steps):
            if batch and batch < n:
                idx = torch.randperm(n, generator=g)[:batch].cuda()
                Xb, yb = F[idx].contiguous(), y[idx].contiguous()
            else:
                Xb, yb = F, y
            want = (it % 100 == 0) or it == steps - 1
            loss = self.mlp.train_step(Xb, yb, lr, want_loss=want)
            if want:
                hist.append(loss)
        return hist

    def predict(self, F: torch.Tensor, fallback_s: int, min_conf: float = 0.6):
        """Per-block slice counts; rows whose top probability is below min_conf get fallback_s."""
        probs = self.mlp.forward(F).cpu().numpy()
        s = probs.argmax(axis=1) + 1
        conf = probs.max(axis=1)
        low = conf < min_conf
        s = np.where(low, fallback_s, s)
        return s.astype(int), conf, int(low.sum())


def evaluate(err: np.ndarray, kmax: float, tau: float, s_pred: np.ndarray):
    """Work and recomputes of per-block counts against the best uniform count at the same budget."""
    nblk = err.shape[0]
    budget = tau * kmax / nblk
    lab = labels_from_errors(err, kmax, tau)
    s_uniform = int(lab.max())
    miss = np.array([err[b, s_pred[b] - 1] > budget for b in range(nblk)])
    s_final = np.where(miss, np.maximum(s_pred, s_uniform), s_pred)
    return {"work_pred": int(sum(pairs(int(x)) for x in s_final)), "work_uniform": nblk * pairs(s_uniform),
            "work_rule": nblk * pairs(rule_slices(tau)), "recomputed": int(miss.sum()), "s_uniform": s_uniform,
            "s_final": [int(x) for x in s_final], "labels": [int(x) for x in lab]}
