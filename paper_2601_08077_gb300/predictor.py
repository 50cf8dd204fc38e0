"""Learned per-block slice counts for the exchange build: training data and training.

The network (16 block features -> 64 -> 64 -> 8 slice counts) runs and trains
on the device through libdf's own kernels; at run time the library itself
predicts, falls back to the rule's count on low confidence and checks the
counts (df_build_K with nslices = LEARNED, after df_set_predictor).  This
module only builds the training set and drives the training steps.

Labels come from the method itself, against FP64: for every 128-function
auxiliary block b the K_b error of the emulated build at every slice count
(df_block_errors), and, per Table 1 level L with count s_L, the per-block
counts with the fewest slice pairs whose summed block errors stay within the
rule's own: sum_b err_b(s_b) <= sum_b err_b(s_L).  The network thereby
serves the accuracy the rule itself achieves at that level, and can only
save work by trading: more slices on blocks whose errors dominate, fewer on
blocks whose errors are negligible.
"""
from __future__ import annotations

import numpy as np
import torch

from . import df

# Table 1: printed accuracy and INT8 count of levels 4..1
LEVELS = {4: (1.2e-7, 3), 3: (4.7e-10, 4), 2: (1.8e-12, 5), 1: (7.1e-15, 6)}
PAIRS = np.array([s * (s + 1) // 2 for s in range(1, 9)])


def pairs(s):
    return s * (s + 1) // 2


def labels_at_rule_accuracy(err: np.ndarray, s_rule: int) -> np.ndarray:
    """Per-block counts (1..8) with few slice pairs and sum_b err[b, s_b - 1] <= sum_b err[b, s_rule - 1].

    Lagrangian relaxation: for a multiplier lam every block independently takes
    argmin_s pairs(s) + lam err[b, s - 1]; the candidates are the assignments at
    every breakpoint lam where some block's choice changes, plus the rule's own
    counts; the feasible candidate with the fewest pairs is then lowered block
    by block (smallest added error first) while it stays feasible.
    """
    err = np.asarray(err, dtype=np.float64)
    nblk = err.shape[0]
    budget = float(err[:, s_rule - 1].sum())
    best = np.full(nblk, s_rule, dtype=np.int64)
    best_work = int(PAIRS[best - 1].sum())
    lams = []
    for b in range(nblk):
        for s1 in range(8):
            for s2 in range(s1 + 1, 8):
                de = err[b, s1] - err[b, s2]
                if de > 0:
                    lams.append((PAIRS[s2] - PAIRS[s1]) / de)
    rev = err[:, ::-1]
    for lam in sorted(set(lams)):
        cost = PAIRS[::-1][None, :] + lam * rev            # reversed: ties go to the larger count
        s = 8 - np.argmin(cost, axis=1)
        e = float(err[np.arange(nblk), s - 1].sum())
        w = int(PAIRS[s - 1].sum())
        if e <= budget and w < best_work:
            best, best_work = s.astype(np.int64), w
    used = float(err[np.arange(nblk), best - 1].sum())
    improved = True
    while improved:
        improved = False
        order = sorted((err[b, best[b] - 2] - err[b, best[b] - 1], b) for b in range(nblk) if best[b] > 1)
        for add, b in order:
            if used + add <= budget:
                best[b] -= 1
                used += add
                improved = True
                break
    return best


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


def molecule_dataset(ctx, C, seed=0, levels=(4, 3, 2, 1)):
    """Features and labels of every block of one molecule at every level.

    The density-change and energy-change features are drawn log-uniformly over
    the range an SCF-like sequence visits (the labels do not depend on them).
    Returns (F [n, 16] float32, labels - 1 [n] int32 on the device, err, kmax).
    """
    rng = np.random.default_rng(seed)
    err, kmax = df.block_errors(ctx, C)
    Fs, ys = [], []
    for level in levels:
        tau, s_rule = LEVELS[level]
        dD = 10.0 ** rng.uniform(-14, 0)
        dE = 10.0 ** rng.uniform(-16, -2)
        Fs.append(df.block_features(ctx, C.shape[1], tau, dD, dE, s_rule))
        lab = labels_at_rule_accuracy(err, s_rule)
        ys.append(torch.from_numpy(lab - 1).to(torch.int32).cuda())
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

    def attach(self, ctx, min_conf: float = 0.6):
        """Let ctx.build_K(C, df.LEARNED) use this network."""
        ctx.set_predictor(self.mlp, min_conf)
