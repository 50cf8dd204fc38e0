"""The adaptive-precision exchange build along an SCF-like sequence of densities.

Section 3.2's scheme on a synthetic sequence: iteration k uses orbitals C_k
whose density differs from the converged D* by 0.1 10^-k (Frobenius), the
Table 1 rule (`df_adaptive_next`, monotone, iterations 0 and 1 at level 4)
picks the slice count of iteration k+1 from the relative change of the
energy E_J + E_K, and every iteration's energies are compared with the
native-FP64 build of the same density.  Optionally the learned predictor
picks per-block slice counts for the tolerance of the rule's level, with
blocks that miss their budget recomputed at the rule's count and counted.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import df, inputs
from . import predictor as pred_mod

LEVEL_TAU = {4: 1.2e-7, 3: 4.7e-10, 2: 1.8e-12, 1: 7.1e-15}


def orbital_sequence(C_star: np.ndarray, n_iter: int, seed: int):
    out = []
    for k in range(n_iter):
        Ck, got = inputs.perturbed_orbitals(C_star, k, seed + 100 + k)
        out.append((Ck, got))
    return out


def run(ctx, orbitals, mode="rule", predictor=None, fp64_from_level=-1, check_blocks=False, level0_slices=0):
    """Run the sequence; returns per-iteration records and totals (times in ms, CUDA events)."""
    nao = ctx.nao
    dev = torch.device("cuda")
    J = torch.empty((nao, nao), dtype=torch.float64, device=dev)
    K = torch.empty_like(J)
    K64 = torch.empty_like(J)
    rho = torch.empty(ctx.naux, dtype=torch.float64, device=dev)
    ctx.adaptive_reset(fp64_from_level)
    ctx.adaptive_level0(level0_slices)
    level, s = 4, pred_mod.rule_slices(LEVEL_TAU[4])
    recs = []
    E_hist, D_prev = [], None
    for k, (Ck, dnorm) in enumerate(orbitals):
        Cg = torch.from_numpy(Ck).to(dev)
        D = inputs.density(Ck)
        Dg = torch.from_numpy(D).to(dev)
        dD = float(np.linalg.norm(D - D_prev)) if D_prev is not None else 1.0
        dE = abs((E_hist[-1] - E_hist[-2]) / E_hist[-1]) if len(E_hist) >= 2 else 1.0
        rec = {"k": k, "level": level, "dnorm": dnorm}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        ctx.build_J(Dg, J, rho)
        if mode == "fp64" or s == 0:
            ctx.build_K(Cg, 0, K)
            rec["slices"] = 0
        elif mode == "predictor" and predictor is not None and level > 0:
            tau = LEVEL_TAU[level]
            F = df.block_features(ctx, Ck.shape[1], tau, dD, dE, s)
            s_blk, conf, nfb = predictor.predict(F, fallback_s=s)
            rec.update(slices_per_block=[int(x) for x in s_blk], fallbacks=nfb)
            ctx.build_K_blocks(Cg, s_blk, K)
        else:
            ctx.build_K(Cg, s, K)
            rec["slices"] = s
        E = ctx.energy(Dg, J, K, rho)
        e1.record()
        torch.cuda.synchronize()
        rec["ms"] = e0.elapsed_time(e1)
        if "slices_per_block" in rec and check_blocks:
            err, kmax = df.block_errors(ctx, Cg)
            tau = LEVEL_TAU[level]
            r = pred_mod.evaluate(err, kmax, tau, np.array(rec["slices_per_block"]))
            rec.update(recomputed=r["recomputed"], work_pred=r["work_pred"], work_rule=r["work_rule"],
                       work_uniform=r["work_uniform"])
            if r["recomputed"]:
                ctx.build_K_blocks(Cg, r["s_final"], K)
                E = ctx.energy(Dg, J, K, rho)
        ctx.build_K(Cg, 0, K64)
        E64 = ctx.energy(Dg, J, K64, rho)
        rec["E"] = E[0] + E[2]
        rec["E_fp64"] = E64[0] + E64[2]
        rec["dE_vs_fp64"] = abs(rec["E"] - rec["E_fp64"])
        rec["max_dK_rel"] = float((K - K64).abs().max() / K64.abs().max())
        E_tot = E[0] + E[2]
        level, s = ctx.adaptive_next(E_tot)
        E_hist.append(E_tot)
        D_prev = D
        recs.append(rec)
    return recs
