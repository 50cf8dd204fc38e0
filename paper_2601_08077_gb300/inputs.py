"""Seeded synthetic inputs for the density-fitting J/K hot path.

This module is the input generator shared by the CUDA path, the tests and the
benchmark.  It draws geometries, basis exponents and orbitals, and it
synthesises the DF tensor B of Eq. cderi (Section 2.1) from closed-form
s-type Gaussian integrals.  It holds none of the hot-path arithmetic (no
split, no slice products, no rho/J/K): those live in the CUDA library and,
independently, in the CPU oracle.

Recipe (the paper's molecules and basis sets are not available, so these
stand in for Table 3's systems, which have N_aux/N_bf = 1.9-4.6 and
N_occ/N_bf = 0.07-0.16):

* geometry: ``n`` atoms drawn one by one, uniform in a cube of edge
  ``L = 10 (n/20)^{1/3}`` bohr (constant atom density), rejecting any draw
  closer than 1.5 bohr to an accepted atom; numpy PCG64 ``default_rng(seed)``;
* basis: per atom 5 AO exponents geometric in [0.1, 10] and 15 auxiliary
  exponents geometric in [0.05, 20], atom-major, normalised primitives;
* B = L^{-1} (P|mu nu) with L L^T = (P|Q) (Eq. cderi), via LAPACK's Cholesky
  and triangular solve;
* orbitals: C = Q factor of the reduced QR of a seeded N(0,1) nao x nocc
  matrix, D = 2 C C^T;
* SCF-like sequence: orbitals perturbed off span(C*) so that
  ||D_k - D*||_F = 0.1 * 10^-k;
* chain molecules (the paper's alkanes are chains): ``n`` atoms along x with
  spacings uniform in [1.6, 2.2] bohr and transverse offsets uniform in
  [-0.4, 0.4] bohr, with Schwarz screening (Section 2.1) of the AO pairs: pair
  (mu, nu) is dropped when sqrt((mu nu|mu nu) max_P (P|P)) < tau, which zeroes
  (P|mu nu) for every P and so B_Pmunu (the contraction of Eq. cderi runs
  over the auxiliary index only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SRC = os.path.join(_HERE, "csrc", "gen_integrals.c")
_GEN_LIB = os.path.join(_HERE, "_build", "libdfgen.so")

AO_EXPONENTS = np.geomspace(0.1, 10.0, 5)
AUX_EXPONENTS = np.geomspace(0.05, 20.0, 15)
MIN_SEPARATION = 1.5
AUX_BLOCK = 128  # auxiliary functions per block (Eqs. df-k-blk-1/2)


def build_generator_library(force: bool = False) -> str:
    """Compile the C integral generator (host code) into ``_build/``."""
    if force or not os.path.exists(_GEN_LIB) or (
            os.path.getmtime(_GEN_LIB) < os.path.getmtime(_GEN_SRC)):
        os.makedirs(os.path.dirname(_GEN_LIB), exist_ok=True)
        tmp = _GEN_LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", _GEN_SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


_lib = None


def _genlib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_generator_library())
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.gen_int3c.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp]
        _lib.gen_metric.argtypes = [ctypes.c_int, dp, dp, dp]
        _lib.gen_oneel.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, dp, dp, dp, dp]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Molecule:
    n_atoms: int
    seed: int
    edge: float
    xyz: np.ndarray                      # [n_atoms, 3] bohr
    ao_xyz: np.ndarray = field(repr=False)
    ao_exp: np.ndarray = field(repr=False)
    aux_xyz: np.ndarray = field(repr=False)
    aux_exp: np.ndarray = field(repr=False)

    @property
    def nao(self) -> int:
        return len(self.ao_exp)

    @property
    def naux(self) -> int:
        return len(self.aux_exp)


def default_edge(n_atoms: int) -> float:
    return 10.0 * (n_atoms / 20.0) ** (1.0 / 3.0)


def geometry(n_atoms: int, seed: int, edge: float) -> np.ndarray:
    rng = np.random.default_rng(seed)
    pts = np.empty((0, 3))
    tries = 0
    while len(pts) < n_atoms:
        p = rng.uniform(0.0, edge, 3)
        tries += 1
        if tries > 1000 * n_atoms + 10000:
            raise RuntimeError("geometry: cannot place %d atoms in a %.2f bohr cube" % (n_atoms, edge))
        if len(pts) == 0 or np.min(np.sqrt(((pts - p) ** 2).sum(1))) >= MIN_SEPARATION:
            pts = np.vstack([pts, p])
    return pts


def molecule(n_atoms: int, seed: int, edge: float | None = None) -> Molecule:
    edge = default_edge(n_atoms) if edge is None else float(edge)
    xyz = geometry(n_atoms, seed, edge)
    return Molecule(
        n_atoms=n_atoms, seed=seed, edge=edge, xyz=xyz,
        ao_xyz=np.ascontiguousarray(np.repeat(xyz, len(AO_EXPONENTS), axis=0)),
        ao_exp=np.tile(AO_EXPONENTS, n_atoms),
        aux_xyz=np.ascontiguousarray(np.repeat(xyz, len(AUX_EXPONENTS), axis=0)),
        aux_exp=np.tile(AUX_EXPONENTS, n_atoms))


def chain_molecule(n_atoms: int, seed: int) -> Molecule:
    """n atoms along x: spacings uniform in [1.6, 2.2] bohr, transverse offsets in [-0.4, 0.4]."""
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.uniform(1.6, 2.2, n_atoms))
    x -= x[0]
    xyz = np.column_stack([x, rng.uniform(-0.4, 0.4, (n_atoms, 2))])
    return Molecule(
        n_atoms=n_atoms, seed=seed, edge=float(x[-1]), xyz=xyz,
        ao_xyz=np.ascontiguousarray(np.repeat(xyz, len(AO_EXPONENTS), axis=0)),
        ao_exp=np.tile(AO_EXPONENTS, n_atoms),
        aux_xyz=np.ascontiguousarray(np.repeat(xyz, len(AUX_EXPONENTS), axis=0)),
        aux_exp=np.tile(AUX_EXPONENTS, n_atoms))


def schwarz_pairs(mol: Molecule, tau: float) -> np.ndarray:
    """Kept AO pairs of Schwarz screening (Section 2.1): sqrt((mu nu|mu nu) max_P (P|P)) >= tau.

    For normalised s primitives, (ab|ab) = (N_a N_b K_ab)^2 2 pi^(5/2) / (p^2 sqrt(2 p))
    with p = a + b (the Coulomb integral of a Gaussian product with itself, F0(0) = 1),
    and (P|P) = N_c^2 2 pi^(5/2) / (c^2 sqrt(2 c)).  Returns a symmetric bool [nao, nao]."""
    a = mol.ao_exp
    p = a[:, None] + a[None, :]
    R2 = np.sum((mol.ao_xyz[:, None, :] - mol.ao_xyz[None, :, :]) ** 2, axis=-1)
    n = (2.0 * a / np.pi) ** 0.75
    nab = n[:, None] * n[None, :] * np.exp(-a[:, None] * a[None, :] / p * R2)
    abab = nab ** 2 * 2.0 * np.pi ** 2.5 / (p * p * np.sqrt(2.0 * p))
    c = mol.aux_exp
    pp = np.max((2.0 * c / np.pi) ** 1.5 * 2.0 * np.pi ** 2.5 / (c * c * np.sqrt(2.0 * c)))
    return np.sqrt(abab * pp) >= tau


def int3c(mol: Molecule) -> np.ndarray:
    out = np.empty((mol.naux, mol.nao, mol.nao))
    _genlib().gen_int3c(mol.nao, mol.naux, _ptr(mol.ao_xyz), _ptr(mol.ao_exp),
                        _ptr(mol.aux_xyz), _ptr(mol.aux_exp), _ptr(out))
    return out


def metric(mol: Molecule) -> np.ndarray:
    out = np.empty((mol.naux, mol.naux))
    _genlib().gen_metric(mol.naux, _ptr(mol.aux_xyz), _ptr(mol.aux_exp), _ptr(out))
    return out


def nuclear_charges(mol: Molecule, Z: float = 2.0) -> np.ndarray:
    """Charge Z on every atom (2: a closed-shell He-like cluster, nocc = n_atoms)."""
    return np.full(mol.n_atoms, float(Z))


def one_electron(mol: Molecule, Z: np.ndarray):
    """Overlap S, kinetic T and nuclear attraction V over the AO primitives
    (for an SCF loop around the build) and the nuclear repulsion energy."""
    n = mol.nao
    S, T, V = np.empty((n, n)), np.empty((n, n)), np.empty((n, n))
    Zc = np.ascontiguousarray(Z, dtype=np.float64)
    _genlib().gen_oneel(n, _ptr(mol.ao_xyz), _ptr(mol.ao_exp), mol.n_atoms, _ptr(mol.xyz), _ptr(Zc),
                        _ptr(S), _ptr(T), _ptr(V))
    R = np.sqrt(np.sum((mol.xyz[:, None, :] - mol.xyz[None, :, :]) ** 2, axis=-1))
    iu = np.triu_indices(mol.n_atoms, 1)
    E_nuc = float(np.sum(Zc[iu[0]] * Zc[iu[1]] / R[iu]))
    return S, T, V, E_nuc


def df_tensor(mol: Molecule, tau: float = 0.0) -> np.ndarray:
    """B[P, mu, nu] = sum_Q L^{-1}[P, Q] (Q|mu nu), L L^T = (P|Q) (Eq. cderi), from the
    Schwarz-screened integrals when tau > 0 (screened pairs are exact zeros in every B_P)."""
    import scipy.linalg as sl
    from scipy.linalg.blas import dtrsm
    V = metric(mol)
    L = sl.cholesky(V, lower=True, check_finite=False)
    T = screened_int3c(mol, tau).reshape(mol.naux, -1)
    # B^T = T^T L^{-T}: a right-side solve on the Fortran-order view of T (no copy)
    Bt = dtrsm(1.0, L, T.T, side=1, lower=1, trans_a=1, overwrite_b=1)
    B = np.ascontiguousarray(Bt.T).reshape(mol.naux, mol.nao, mol.nao)
    # every B_P is symmetric in (mu, nu); make it so bit for bit whatever the BLAS did
    for P in range(mol.naux):
        B[P] = 0.5 * (B[P] + B[P].T)
    return B


def pack_upper(B: np.ndarray) -> np.ndarray:
    """Each B_P's upper triangle row by row: [naux, nao (nao + 1) / 2] (df_setup_packed's layout)."""
    naux, nao, _ = B.shape
    iu = np.triu_indices(nao)
    return np.ascontiguousarray(B[:, iu[0], iu[1]])


def leading_aux(mol: Molecule, nrows: int) -> Molecule:
    """The same molecule with only its first nrows auxiliary functions."""
    if nrows >= mol.naux:
        return mol
    return Molecule(mol.n_atoms, mol.seed, mol.edge, mol.xyz, mol.ao_xyz, mol.ao_exp,
                    np.ascontiguousarray(mol.aux_xyz[:nrows]), np.ascontiguousarray(mol.aux_exp[:nrows]))


def df_tensor_rows(mol: Molecule, nrows: int) -> np.ndarray:
    """The first nrows auxiliary rows of B (Eq. cderi), without forming the rest.

    Forward substitution makes row P of L^{-1} T depend only on rows <= P, and
    the leading block of the Cholesky factor is the factor of the leading block
    of the metric, so B[:nrows] needs only the first nrows auxiliary functions.
    Equal to df_tensor(mol)[:nrows] up to the solver's rounding.
    """
    import scipy.linalg as sl
    from scipy.linalg.blas import dtrsm
    nrows = min(nrows, mol.naux)
    sub = Molecule(mol.n_atoms, mol.seed, mol.edge, mol.xyz, mol.ao_xyz, mol.ao_exp,
                   np.ascontiguousarray(mol.aux_xyz[:nrows]), np.ascontiguousarray(mol.aux_exp[:nrows]))
    L = sl.cholesky(metric(sub), lower=True, check_finite=False)
    T = int3c(sub).reshape(nrows, -1)
    Bt = dtrsm(1.0, L, T.T, side=1, lower=1, trans_a=1, overwrite_b=1)
    B = np.ascontiguousarray(Bt.T).reshape(nrows, mol.nao, mol.nao)
    for P in range(nrows):
        B[P] = 0.5 * (B[P] + B[P].T)
    return B


def _preload_torch_linalg():
    """Load torch's CUDA linear-algebra library by absolute path.  torch opens
    it lazily by bare name, which fails in processes whose library search path
    has been changed (a profiler's injection, for one)."""
    import ctypes
    import torch
    path = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(path):
        ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)


def df_tensor_device(mol: Molecule, device="cuda", nrows: int | None = None):
    """B of Eq. cderi with the triangular solve on a CUDA device (torch / cuBLAS).

    Input synthesis for the large workloads (batches, predictor training, the
    240-atom molecule): the integrals and the metric's Cholesky factor are
    formed on the host as in ``df_tensor``, the solve L B = (P|mu nu) runs on
    the device.  The result agrees with ``df_tensor`` to the conditioning of
    the metric, not bit for bit, so parity tests use ``df_tensor``.  With
    ``nrows`` only the first nrows auxiliary rows are formed (as in
    ``df_tensor_rows``: the forward substitution needs no later rows).
    Returns a contiguous float64 tensor [naux or nrows, nao, nao] on ``device``.
    """
    import scipy.linalg as sl
    import torch
    _preload_torch_linalg()
    if nrows is not None and nrows < mol.naux:
        mol = Molecule(mol.n_atoms, mol.seed, mol.edge, mol.xyz, mol.ao_xyz, mol.ao_exp,
                       np.ascontiguousarray(mol.aux_xyz[:nrows]), np.ascontiguousarray(mol.aux_exp[:nrows]))
    V = metric(mol)
    L = torch.from_numpy(sl.cholesky(V, lower=True, check_finite=False)).to(device)
    T = torch.from_numpy(int3c(mol).reshape(mol.naux, -1)).to(device)
    B = torch.linalg.solve_triangular(L, T, upper=False)
    del T
    B = B.reshape(mol.naux, mol.nao, mol.nao).contiguous()
    for p0 in range(0, mol.naux, 256):   # exact symmetry per P, in chunks
        Bc = B[p0:p0 + 256]
        Bc.copy_(0.5 * (Bc + Bc.transpose(1, 2)))
    return B


def orbitals(nao: int, nocc: int, seed: int) -> np.ndarray:
    """Orthonormal occupied coefficients C [nao, nocc] (QR of seeded N(0,1))."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((nao, nocc)))
    return np.ascontiguousarray(q)


def density(C: np.ndarray) -> np.ndarray:
    """D = 2 C C^T, symmetric bit for bit."""
    D = 2.0 * C @ C.T
    return 0.5 * (D + D.T)


def perturbed_orbitals(C_star: np.ndarray, k: int, seed: int, base: float = 0.1) -> tuple[np.ndarray, float]:
    """Orbitals C_k of the SCF-like sequence: ||2 C_k C_k^T - D*||_F ~= base*10^-k.

    C_k is the Q factor of C* + t Z with Z seeded N(0,1) projected off
    span(C*); t is rescaled by a few secant steps so that the density change
    hits its target.  Returns (C_k, achieved norm).
    """
    nao, nocc = C_star.shape
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((nao, nocc))
    Z -= C_star @ (C_star.T @ Z)
    Z /= np.linalg.norm(Z)
    D_star = density(C_star)
    target = base * 10.0 ** (-k)

    def dnorm(t):
        q, _ = np.linalg.qr(C_star + t * Z)
        return q, np.linalg.norm(density(q) - D_star)

    t = target / (2.0 * np.sqrt(2.0))   # ||dD|| ~ 2 sqrt(2) t for small t
    q, got = dnorm(t)
    for _ in range(3):
        if got <= 0 or not np.isfinite(got):
            break
        t *= target / got
        q, got = dnorm(t)
    return np.ascontiguousarray(q), float(got)


def aux_blocks(naux: int, block: int = AUX_BLOCK) -> list[tuple[int, int]]:
    return [(p0, min(p0 + block, naux)) for p0 in range(0, naux, block)]


# --- the workloads -----------------------------------------------------------

@dataclass
class Workload:
    name: str
    n_atoms: int
    nocc: int
    seed: int
    shape: str = "cube"     # "cube": constant-density cube; "chain": the chain geometry
    tau: float = 0.0        # Schwarz screening threshold of the AO pairs (0: none)

    @property
    def nao(self):
        return 5 * self.n_atoms

    @property
    def naux(self):
        return 15 * self.n_atoms


# One molecule of 20 atoms (nao 100, naux 300, nocc 20): plain FP64 J/K.
SMALL = Workload("df-20atom-nao100-naux300-nocc20", 20, 20, 1000 * 0 + 0)
# One molecule of 120 atoms (nao 600, naux 1800, nocc 120): fixed-slice sweep.
MEDIUM = Workload("df-120atom-nao600-naux1800-nocc120", 120, 120, 1000 * 1 + 0)
# One molecule of 240 atoms (nao 1200, naux 3600, nocc 250): adaptive sequence.
LARGE = Workload("df-240atom-nao1200-naux3600-nocc250", 240, 250, 1000 * 2 + 0)


# A 240-atom chain with the 240-atom molecule's sizes (nao 1200, naux 3600, nocc 250)
# and Schwarz screening at 1e-12: about 5 % of the AO pairs survive (block-sparse B).
CHAIN = Workload("df-chain240-nao1200-naux3600-nocc250-scr1e-12", 240, 250, 1000 * 7 + 0, "chain", 1e-12)


def workload_molecule(w: Workload) -> Molecule:
    return chain_molecule(w.n_atoms, w.seed) if w.shape == "chain" else molecule(w.n_atoms, w.seed)


def screened_int3c(mol: Molecule, tau: float) -> np.ndarray:
    """(P|mu nu) with the Schwarz-screened pairs set to zero for every P (tau 0: none)."""
    T = int3c(mol)
    if tau > 0.0:
        T[:, ~schwarz_pairs(mol, tau)] = 0.0
    return T


# 60 atoms with the 120-atom molecule's occupied count: the same tile shapes in a
# few GB of device memory (used for counter captures).
PROFILE = Workload("df-60atom-nao300-naux900-nocc120", 60, 120, 1000 * 9 + 0)


def batch_workloads(n_mol: int = 48, seed: int = 3000) -> list[Workload]:
    """Grouped batch: atom counts uniform in [30, 120], nocc = nao/5."""
    rng = np.random.default_rng(seed)
    atoms = rng.integers(30, 121, size=n_mol)
    return [Workload("batch-%02d" % i, int(a), int(a), seed + 1 + i) for i, a in enumerate(atoms)]


def training_workloads(n_mol: int = 200, seed: int = 4000) -> list[Workload]:
    """Predictor training set: nao 100..600 (20..120 atoms), nocc = nao/5."""
    rng = np.random.default_rng(seed)
    atoms = rng.integers(20, 121, size=n_mol)
    return [Workload("train-%03d" % i, int(a), int(a), seed + 1 + i) for i, a in enumerate(atoms)]


def make_inputs(w: Workload):
    """(molecule, B, C, D) for a workload; orbitals use seed+1."""
    mol = molecule(w.n_atoms, w.seed)
    B = df_tensor(mol)
    C = orbitals(mol.nao, w.nocc, w.seed + 1)
    return mol, B, C, density(C)
