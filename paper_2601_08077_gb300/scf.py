"""Restricted Hartree-Fock around the DF J/K build, with the precision of the
exchange build chosen every iteration by the paper's rule (Section 3.2,
Table 1) from the relative change of the true SCF energy.

Each iteration: diagonalise the Fock matrix in the canonically orthogonalised
basis (cuSOLVER through torch), form C_occ and D = 2 C_occ C_occ^T, build J
(FP64) and K (INT8 slices at the rule's count, or FP64) with libdf, form
F = h + J - K (K without the occupation factor: the usual exchange matrix
2K enters with -1/2), E = tr(D h) + 1/2 tr(D J) - 1/2 tr(D K) + E_nuc, and
extrapolate F by DIIS on the commutator F D S - S D F.  The rule is monotone
(no return to fewer slices) and its level 0 is native FP64 or, on GB300,
optionally 8 slices (`level0_slices`).
"""
from __future__ import annotations

import numpy as np
import torch

from . import df


def _orthogonaliser(S: torch.Tensor, threshold: float = 1e-7) -> torch.Tensor:
    s, U = torch.linalg.eigh(S)
    keep = s > threshold * s[-1]
    return U[:, keep] / torch.sqrt(s[keep])[None, :]


def _diis(Fs, errs):
    """Pulay's DIIS: the combination of the stored F minimising |sum c_i e_i|
    under sum c_i = 1 (a bordered linear system)."""
    n = len(Fs)
    E = torch.stack([e.reshape(-1) for e in errs])
    Bm = torch.full((n + 1, n + 1), -1.0, dtype=torch.float64, device=E.device)
    Bm[:n, :n] = E @ E.T
    Bm[n, n] = 0.0
    rhs = torch.zeros(n + 1, dtype=torch.float64, device=E.device)
    rhs[n] = -1.0
    c = torch.linalg.solve(Bm, rhs)[:n]
    return torch.einsum("i,ijk->jk", c, torch.stack(Fs))


def run(ctx, h, S, nocc: int, E_nuc: float, mode: str = "rule", level0_slices: int = 0, fixed_slices: int = 3,
        maxiter: int = 60, e_tol: float = 1e-10, d_tol: float = 1e-7, ndiis: int = 8, device="cuda"):
    """SCF on the context's B.  mode: 'rule' (Table 1), 'fp64' (every K in
    FP64) or 'fixed' (every K at `fixed_slices`, the fixed-level runs the
    paper contrasts with the rule in Section 4).  Returns per-iteration
    records (level, slices, E, dE, ms of the J/K build and energies) and the
    final energy."""
    dev = torch.device(device)
    h = torch.as_tensor(h, dtype=torch.float64, device=dev)
    S = torch.as_tensor(S, dtype=torch.float64, device=dev)
    X = _orthogonaliser(S)
    F = h.clone()
    J = torch.empty_like(h)
    K = torch.empty_like(h)
    rho = torch.empty(ctx.naux, dtype=torch.float64, device=dev)
    ctx.adaptive_reset()
    ctx.adaptive_level0(level0_slices)
    level, s = 4, df.level_slices(4)
    Fs, errs, recs = [], [], []
    E_old = None
    converged = False
    for it in range(maxiter):
        _, Cp = torch.linalg.eigh(X.T @ F @ X)
        C_occ = (X @ Cp[:, :nocc]).contiguous()
        D = 2.0 * C_occ @ C_occ.T
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ns = {"fp64": 0, "fixed": fixed_slices}.get(mode, s)
        ctx.build_JK(D, C_occ, ns, J, rho, K)
        EJ, _, EK = ctx.energy(D, J, K, rho)
        e1.record()
        torch.cuda.synchronize()
        E = float(torch.sum(D * h)) + EJ + EK + E_nuc
        Fk = h + J - K
        err = Fk @ D @ S - S @ D @ Fk
        recs.append({"it": it, "level": level if mode == "rule" else 0, "slices": ns, "E": E,
                     "dE": None if E_old is None else E - E_old, "ms": e0.elapsed_time(e1),
                     "comm": float(err.abs().max())})
        if E_old is not None and abs(E - E_old) < e_tol and float(err.abs().max()) < d_tol:
            converged = True
            break
        E_old = E
        if mode == "rule":
            level, s = ctx.adaptive_next(E)
        Fs.append(Fk)
        errs.append(X.T @ err @ X)
        Fs, errs = Fs[-ndiis:], errs[-ndiis:]
        F = _diis(Fs, errs) if len(Fs) > 1 else Fk
    ctx.sync_status()
    return {"E": recs[-1]["E"], "converged": converged, "iterations": recs}
