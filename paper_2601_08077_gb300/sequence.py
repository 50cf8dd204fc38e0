"""The adaptive-precision exchange build along an SCF-like sequence of densities.

Section 3.2's scheme on a synthetic sequence: iteration k uses orbitals C_k
whose density differs from the converged D* by 0.1 10^-k (Frobenius).  The
library's controller (df_adaptive_next: Table 1, monotone, iterations 0 and 1
at level 4) picks each iteration's level from the relative change of the
energy E_J + E_K; J and K of an iteration come from one df_build_JK call
(rho and J beside the X split), at that level's count (mode "rule", ADAPTIVE), with per-block counts from the attached network
(mode "learned", LEARNED: prediction, fallback, check and recompute all in
the library), or in native FP64 (mode "fp64").  Optionally every iteration's
K and energy are compared with the native-FP64 build of the same density
(outside the timed region).
"""
from __future__ import annotations

import numpy as np
import torch

from . import df, inputs


def orbital_sequence(C_star: np.ndarray, n_iter: int, seed: int):
    out = []
    for k in range(n_iter):
        Ck, got = inputs.perturbed_orbitals(C_star, k, seed + 100 + k)
        out.append((Ck, got))
    return out


def run(ctx, orbitals, mode="rule", fp64_from_level=-1, level0_slices=0, compare_fp64=True, fp64_cache=None):
    """Run the sequence; returns per-iteration records (times in ms, CUDA events).

    compare_fp64: True every iteration, "last" the last one only, False none.
    fp64_cache (a dict, optional) keeps each iteration's native-FP64 K and energy
    across runs over the same orbitals, so the comparison build runs once."""
    nao = ctx.nao
    dev = torch.device("cuda")
    J = torch.empty((nao, nao), dtype=torch.float64, device=dev)
    K = torch.empty_like(J)
    rho = torch.empty(ctx.naux, dtype=torch.float64, device=dev)
    ctx.adaptive_reset(fp64_from_level)
    ctx.adaptive_level0(level0_slices)
    nslices = {"rule": df.ADAPTIVE, "learned": df.LEARNED, "fp64": 0}[mode]
    recs = []
    for k, (Ck, dnorm) in enumerate(orbitals):
        Cg = torch.from_numpy(Ck).to(dev)
        Dg = torch.from_numpy(inputs.density(Ck)).to(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        _, _, _, st = ctx.build_JK(Dg, Cg, nslices, J, rho, K)
        E = ctx.energy(Dg, J, K, rho)
        e1.record()
        torch.cuda.synchronize()
        rec = {"k": k, "dnorm": dnorm, "ms": e0.elapsed_time(e1), "E": E[0] + E[2], **st.as_dict()}
        if compare_fp64 is True or (compare_fp64 == "last" and k == len(orbitals) - 1):
            if fp64_cache is not None and k in fp64_cache:
                K64, E64 = fp64_cache[k]
            else:
                K64 = torch.empty_like(J)
                ctx.build_K(Cg, 0, K64)
                E64 = ctx.energy(Dg, J, K64, rho)
                if fp64_cache is not None:
                    fp64_cache[k] = (K64, E64)
            rec["E_fp64"] = E64[0] + E64[2]
            rec["dE_vs_fp64"] = abs(rec["E"] - rec["E_fp64"])
            rec["max_dK_rel"] = float((K - K64).abs().max() / K64.abs().max())
        ctx.adaptive_next(rec["E"])
        recs.append(rec)
    return recs
