"""CPU oracle for a restricted Hartree-Fock loop around the DF J/K build.

TEST INFRASTRUCTURE ONLY (tests/, smoke(), bench.py's CPU legs may import it;
the CUDA library never does).  Plain NumPy in FP64.

The paper drives its adaptive precision by the energy change of real SCF
iterations (Section 3.2, Table 1).  This module gives that loop for the
synthetic molecules: one-electron integrals over normalised s Gaussians
(overlap, kinetic energy, attraction to nuclei of charge Z), the RHF Fock
matrix with density-fitted J and K, F = h + J - K (K without the occupation
factor: for D = 2 C C^T the usual exchange matrix is 2K, entering with -1/2),
the energy E = tr(D h) + 1/2 tr(D J) - 1/2 tr(D K) + E_nuc, canonical
orthogonalisation of the overlap, and DIIS on the commutator F D S - S D F.

Pins (tests/test_oracle_scf.py): S_aa = 1; T_aa = 3a/2; a normalised s
Gaussian at a nucleus of charge Z feels -2 Z sqrt(2a/pi); S, T, V symmetric,
S and T positive definite; the SCF energy of a He-like system in a
one-function basis (one auxiliary function fits it exactly) against its
closed form 2h + (aa|aa); the converged Fock matrix commutes with the
density (F D S = S D F); the converged D is idempotent in the S metric and
holds the electron count; the SCF energy lies below the first iteration's.
"""
from __future__ import annotations

import math

import numpy as np

from . import df_oracle as O

PI = math.pi


def gaussian_pairs(ao_xyz, ao_exp):
    a = np.asarray(ao_exp, dtype=np.float64)
    p, Pc, Kab = O.gaussian_product(a[:, None], ao_xyz[:, None, :], a[None, :], ao_xyz[None, :, :])
    nn = O.norm_s(a)[:, None] * O.norm_s(a)[None, :]
    return a, p, Pc, Kab, nn


def overlap(ao_xyz, ao_exp):
    """S_ab = N_a N_b (pi/p)^{3/2} exp(-ab/p |A-B|^2)."""
    a, p, _, Kab, nn = gaussian_pairs(ao_xyz, ao_exp)
    return nn * (PI / p) ** 1.5 * Kab


def kinetic(ao_xyz, ao_exp):
    """T_ab = <a| -1/2 nabla^2 |b> = (ab/p) (3 - 2 (ab/p) |A-B|^2) S_ab."""
    a, p, _, Kab, nn = gaussian_pairs(ao_xyz, ao_exp)
    mu = a[:, None] * a[None, :] / p
    R2 = np.sum((ao_xyz[:, None, :] - ao_xyz[None, :, :]) ** 2, axis=-1)
    return mu * (3.0 - 2.0 * mu * R2) * nn * (PI / p) ** 1.5 * Kab


def nuclear(ao_xyz, ao_exp, nuc_xyz, Z):
    """V_ab = -sum_C Z_C N_a N_b (2 pi/p) exp(-ab/p |A-B|^2) F0(p |P-C|^2)."""
    a, p, Pc, Kab, nn = gaussian_pairs(ao_xyz, ao_exp)
    V = np.zeros_like(p)
    for C, z in zip(nuc_xyz, Z):
        R2 = np.sum((Pc - C[None, None, :]) ** 2, axis=-1)
        V -= z * O.boys_f0(p * R2)
    return nn * (2.0 * PI / p) * Kab * V


def nuclear_repulsion(nuc_xyz, Z):
    E = 0.0
    for i in range(len(Z)):
        for j in range(i):
            E += Z[i] * Z[j] / float(np.linalg.norm(nuc_xyz[i] - nuc_xyz[j]))
    return E


def orthogonaliser(S, threshold=1e-7):
    """Canonical orthogonalisation: X = U s^{-1/2} over eigenvalues > threshold * max."""
    s, U = np.linalg.eigh(S)
    keep = s > threshold * s[-1]
    return U[:, keep] / np.sqrt(s[keep])[None, :]


def density(C_occ):
    return 2.0 * C_occ @ C_occ.T


def fock_energy(h, D, J, K, E_nuc):
    """F = h + J - K and E = tr(D h) + 1/2 tr(D J) - 1/2 tr(D K) + E_nuc."""
    F = h + J - K
    E = float(np.sum(D * h) + 0.5 * np.sum(D * J) - 0.5 * np.sum(D * K)) + E_nuc
    return F, E


def diis_extrapolate(Fs, errs):
    """Pulay's DIIS: the combination of the stored F minimising |sum c_i e_i|, sum c_i = 1."""
    n = len(Fs)
    Bm = np.empty((n + 1, n + 1))
    for i in range(n):
        for j in range(n):
            Bm[i, j] = float(np.sum(errs[i] * errs[j]))
    Bm[n, :] = -1.0
    Bm[:, n] = -1.0
    Bm[n, n] = 0.0
    rhs = np.zeros(n + 1)
    rhs[n] = -1.0
    c = np.linalg.solve(Bm, rhs)[:n]
    return sum(ci * Fi for ci, Fi in zip(c, Fs))


def scf(h, S, nocc, jk, E_nuc=0.0, maxiter=60, e_tol=1e-10, d_tol=1e-7, ndiis=8):
    """RHF.  jk(C_occ, D) -> (J, K).  Returns dict(E, C, D, F, history, converged)."""
    X = orthogonaliser(S)
    F = h.copy()
    Fs, errs, hist = [], [], []
    E_old = None
    C_occ = D = None
    converged = False
    for it in range(maxiter):
        e, Cp = np.linalg.eigh(X.T @ F @ X)
        C = X @ Cp
        C_occ = C[:, :nocc]
        D = density(C_occ)
        J, K = jk(C_occ, D)
        Fk, E = fock_energy(h, D, J, K, E_nuc)
        err = Fk @ D @ S - S @ D @ Fk
        hist.append(E)
        if E_old is not None and abs(E - E_old) < e_tol and np.max(np.abs(err)) < d_tol:
            F = Fk
            converged = True
            break
        E_old = E
        Fs.append(Fk)
        errs.append(X.T @ err @ X)
        Fs, errs = Fs[-ndiis:], errs[-ndiis:]
        F = diis_extrapolate(Fs, errs) if len(Fs) > 1 else Fk
    return {"E": hist[-1], "C": C_occ, "D": D, "F": F, "history": hist, "converged": converged}


def df_jk(B):
    """The exact DF J and K of the oracle for a fixed B."""
    def jk(C_occ, D):
        rho = O.rho(B, D)
        return O.coulomb(B, rho), O.exchange(B, C_occ)
    return jk
