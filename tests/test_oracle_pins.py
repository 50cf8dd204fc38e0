"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU (no GPU marker).  Each is chosen so that a
plausible mistake in the oracle (a dropped term, a wrong sign, a transposed
operand, a wrong factor of 2, an off-by-one in a digit index) fails it.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl
from scipy.integrate import quad
from scipy.special import erf

from oracle import df_oracle as O
from paper_2601_08077_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- fixtures ---------------------------------------------------------------

@pytest.fixture(scope="module")
def tiny():
    """Two atoms: nao 10, naux 30 (small enough for four-index brute force)."""
    mol = inputs.molecule(2, seed=7, edge=3.0)
    T = O.int3c(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp)
    V = O.metric(mol.aux_xyz, mol.aux_exp)
    B = O.df_tensor(T, V)
    C = inputs.orbitals(mol.nao, 3, seed=8)
    return mol, T, V, B, C, inputs.density(C)


@pytest.fixture(scope="module")
def small():
    """The 20-atom molecule (nao 100, naux 300, nocc 20)."""
    w = inputs.SMALL
    mol = inputs.molecule(w.n_atoms, w.seed)
    B = inputs.df_tensor(mol)
    C = inputs.orbitals(mol.nao, w.nocc, w.seed + 1)
    return mol, B, C, inputs.density(C)


# --- integrals ----------------------------------------------------------------

def test_boys_limits_and_quadrature():
    assert O.boys_f0(np.array([0.0]))[0] == 1.0
    for T in [1e-12, 1e-9, 1e-6, 0.1, 1.0, 7.5, 40.0, 300.0]:
        ref, _ = quad(lambda u: math.exp(-T * u * u), 0.0, 1.0, epsabs=1e-15, epsrel=1e-14)
        assert abs(O.boys_f0(np.array([T]))[0] - ref) < 1e-13
    T = 900.0
    assert abs(O.boys_f0(np.array([T]))[0] - 0.5 * math.sqrt(math.pi / T)) < 1e-15


def test_gaussian_product_theorem():
    rng = np.random.default_rng(1)
    a, b = np.array(0.7), np.array(2.3)
    A, B = rng.normal(size=3), rng.normal(size=3)
    p, P, K = O.gaussian_product(a, A, b, B)
    for r in rng.normal(size=(5, 3)):
        lhs = math.exp(-a * np.sum((r - A) ** 2)) * math.exp(-b * np.sum((r - B) ** 2))
        rhs = K * math.exp(-p * np.sum((r - P) ** 2))
        assert abs(lhs - rhs) <= 1e-14 * max(lhs, 1e-300)


@pytest.mark.parametrize("a,b,R", [(0.3, 0.3, 0.0), (1.0, 4.0, 0.7), (0.05, 20.0, 3.0), (2.0, 0.5, 25.0)])
def test_unit_charge_gaussians_interact_as_erf_over_R(a, b, R):
    """Unit-charge Gaussians (a/pi)^{3/2} e^{-a r^2}: energy erf(sqrt(mu) R)/R, mu = ab/(a+b)."""
    A = np.zeros(3)
    B = np.array([0.0, 0.0, R])
    e = (a / math.pi) ** 1.5 * (b / math.pi) ** 1.5 * O.coulomb_ss(np.array(a), A, np.array(b), B)
    mu = a * b / (a + b)
    ref = 2.0 * math.sqrt(mu / math.pi) if R == 0 else erf(math.sqrt(mu) * R) / R
    assert abs(float(e) - ref) < 1e-14 * max(1.0, ref)
    if R > 20:
        assert abs(float(e) - 1.0 / R) < 1e-12


def test_int3c_reduces_to_metric_when_centres_coincide():
    """(c|ab) with A = B equals N_a N_b / N_{a+b} (c|d) with d = a+b at that centre."""
    rng = np.random.default_rng(2)
    A = rng.normal(size=(1, 3))
    aux_xyz = rng.normal(size=(4, 3))
    aux_exp = np.array([0.1, 0.9, 3.0, 11.0])
    ao_exp = np.array([0.4, 1.3])
    T = O.int3c(np.vstack([A, A]), ao_exp, aux_xyz, aux_exp)
    d = ao_exp.sum()
    V = O.metric(np.vstack([aux_xyz, A]), np.concatenate([aux_exp, [d]]))
    ratio = O.norm_s(ao_exp[0]) * O.norm_s(ao_exp[1]) / O.norm_s(d)
    np.testing.assert_allclose(T[:, 0, 1], ratio * V[:4, 4], rtol=1e-13)


def test_metric_symmetric_positive_definite(small):
    mol = small[0]
    V = O.metric(mol.aux_xyz, mol.aux_exp)
    assert np.array_equal(V, V.T)
    w = sl.eigh(V, eigvals_only=True)
    assert w.min() > 0.0


def test_oracle_integrals_match_generator(small):
    """The generator (C) and the oracle (NumPy) integrals are separate codes."""
    mol = small[0]
    np.testing.assert_allclose(O.metric(mol.aux_xyz, mol.aux_exp), inputs.metric(mol), rtol=1e-13, atol=1e-15)
    T = O.int3c(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp)
    np.testing.assert_allclose(T, inputs.int3c(mol), rtol=1e-12, atol=1e-16)


# --- DF tensor -------------------------------------------------------------------

def test_cholesky_and_solve_match_lapack(tiny):
    """Backward-stable: tiny residuals; forward agreement with LAPACK within the conditioning."""
    _, T, V, B, _, _ = tiny
    L = O.cholesky(V)
    assert np.array_equal(L, np.tril(L))
    assert np.max(np.abs(L @ L.T - V)) <= 1e-14 * np.max(np.abs(V))
    cond = np.linalg.cond(V)
    assert np.max(np.abs(L - np.linalg.cholesky(V))) <= 1e-15 * math.sqrt(cond) * np.max(np.abs(L)) * 10
    Tm = T.reshape(T.shape[0], -1)
    Bm = B.reshape(T.shape[0], -1)
    assert np.max(np.abs(L @ Bm - Tm)) <= 1e-13 * np.max(np.abs(Tm))
    ref = sl.solve_triangular(L, Tm, lower=True)
    assert np.max(np.abs(Bm - ref)) <= 1e-15 * math.sqrt(cond) * np.max(np.abs(ref)) * 10


def test_cholesky_rejects_indefinite():
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_df_tensor_invariant_to_aux_scaling(tiny):
    """Rescaling the auxiliary functions by S > 0 leaves B unchanged (chol(SVS) = S L)."""
    _, T, V, B, _, _ = tiny
    S = np.linspace(0.3, 3.0, V.shape[0])
    B2 = O.df_tensor(T * S[:, None, None], V * S[:, None] * S[None, :])
    # exact in exact arithmetic; the FP64 triangular solves differ within the
    # usual forward-error bound n u cond(L) |B|, cond(L) = sqrt(cond(V))
    n = V.shape[0]
    tol = n * 2.0 ** -52 * math.sqrt(np.linalg.cond(V)) * np.max(np.abs(B))
    assert np.max(np.abs(B2 - B)) <= tol


def test_df_tensor_reproduces_three_centre_integrals(tiny):
    """sum_Q L_PQ B_Q = (P|mn): the fit reproduces its own data."""
    _, T, V, B, _, _ = tiny
    L = O.cholesky(V)
    np.testing.assert_allclose(np.einsum("pq,qmn->pmn", L, B), T, rtol=1e-10, atol=1e-13)


def test_oracle_df_tensor_matches_generator(small):
    mol, B, _, _ = small
    T = O.int3c(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp)
    V = O.metric(mol.aux_xyz, mol.aux_exp)
    Bo = O.df_tensor(T, V)
    assert np.max(np.abs(Bo - B)) < 1e-8 * np.max(np.abs(B))


# --- J, K, energies ------------------------------------------------------------------

def test_J_K_symmetry_and_K_psd(small):
    _, B, C, D = small
    J = O.coulomb(B, O.rho(B, D))
    K = O.exchange(B, C)
    assert np.max(np.abs(J - J.T)) <= 1e-13 * np.max(np.abs(J))
    assert np.max(np.abs(K - K.T)) <= 1e-13 * np.max(np.abs(K))
    assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() > -1e-12 * np.max(np.abs(K))


def test_energies_two_ways(small):
    _, B, C, D = small
    r = O.rho(B, D)
    J = O.coulomb(B, r)
    K = O.exchange(B, C)
    EJ, EK = O.energies(D, J, K)
    EJ2, EK2 = O.energies_alt(B, C, r)
    assert abs(EJ - EJ2) <= 1e-12 * abs(EJ)
    assert abs(EK - EK2) <= 1e-12 * abs(EK)
    assert EJ > 0 > EK


def test_exchange_matches_quadruple_loop(tiny):
    _, _, _, B, C, D = tiny
    Kbf = O.exchange_bruteforce(B, D)
    np.testing.assert_allclose(O.exchange(B, C), 0.5 * Kbf, rtol=1e-12, atol=1e-14)


def test_df_coulomb_energy_is_variational(tiny):
    """Coulomb-metric fitting never overestimates the Coulomb energy, and is close."""
    mol, _, _, B, C, D = tiny
    eri = O.eri4(mol.ao_xyz, mol.ao_exp)
    E_exact = 0.5 * np.einsum("ab,abcd,cd->", D, eri, D)
    r = O.rho(B, D)
    E_df = 0.5 * r @ r
    assert E_df <= E_exact * (1 + 1e-14)
    assert (E_exact - E_df) / E_exact < 1e-2
    # the exact four-index integrals also give the same K up to the fitting error
    K_exact = 0.5 * np.einsum("acbd,cd->ab", eri, D)
    K_df = O.exchange(B, C)
    assert np.max(np.abs(K_exact - K_df)) < 0.05 * np.max(np.abs(K_exact))


# --- INT8 slice emulation -------------------------------------------------------------

def _spread_matrix(rng, m, n, spread=20):
    return rng.standard_normal((m, n)) * np.exp2(rng.integers(-spread, 1, size=(m, n)))


def test_row_exponent_definition():
    A = np.array([[127 / 128 * 4.0, 0.0], [127 / 128 * 4.0 * (1 - 2 ** -52), 1.0], [0.0, 0.0], [-3.0, 1e-300]])
    e = O.row_exponents(A)
    # smallest e with max|row| < 127/128 2^e
    assert list(e) == [3, 2, 0, 2]


def test_split_digit_ranges_and_exact_reconstruction():
    rng = np.random.default_rng(3)
    A = _spread_matrix(rng, 37, 53)
    A[5] = 0.0
    e, d = O.split_rows(A, 8)
    assert d.dtype == np.int8
    assert d.min() >= -128 and d.max() <= 127
    assert np.abs(d[0].astype(int)).max() <= 127
    # all 8 digits give RNE(x 2^63) 2^{e-63} exactly
    rec = O.reconstruct(e, d)
    ref = np.ldexp(np.rint(np.ldexp(A, 63 - e[:, None])), e[:, None] - 63)
    assert np.array_equal(rec, ref)
    # entries within 2^-11 of their row scale carry no bits below 2^-63: exact
    big = np.abs(A) >= np.ldexp(1.0, e[:, None] - 11)
    assert np.array_equal(rec[big], A[big])
    assert np.all(d[:, 5] == 0) and e[5] == 0


def test_split_prefix_truncation_bound():
    rng = np.random.default_rng(4)
    A = _spread_matrix(rng, 20, 40, spread=8)
    e, d = O.split_rows(A, 8)
    for s in range(1, 8):
        rec = O.reconstruct(e, d[:s])
        bound = np.ldexp(1.004 * 2.0 ** (-8 * s) + 2.0 ** -64, e)[:, None]
        assert np.all(np.abs(rec - A) <= bound)


def test_slice_products_match_digit_loops():
    rng = np.random.default_rng(5)
    Ad = rng.integers(-128, 128, size=(4, 3, 7)).astype(np.int8)
    Bd = rng.integers(-128, 128, size=(4, 2, 7)).astype(np.int8)
    S = O.slice_products(Ad, Bd, 4)
    for g in range(4):
        for m in range(3):
            for n in range(2):
                v = 0
                for t in range(4):
                    for u in range(4):
                        if t + u == g:
                            v += sum(int(Ad[t, m, k]) * int(Bd[u, n, k]) for k in range(7))
                assert S[g, m, n] == v


def test_integer_valued_matrices_emulate_exactly():
    rng = np.random.default_rng(6)
    A = rng.integers(-100, 101, size=(9, 31)).astype(float) * np.exp2(rng.integers(-5, 5, size=(9, 1)))
    B = rng.integers(-100, 101, size=(31, 6)).astype(float) * np.exp2(rng.integers(-5, 5, size=(1, 6)))
    for s in (1, 2, 3, 8):
        assert np.array_equal(O.emulated_matmul(A, B, s), A @ B)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 6, 7, 8])
def test_emulation_within_error_bound(s):
    rng = np.random.default_rng(10 + s)
    A = _spread_matrix(rng, 6, 17, spread=12)
    B = _spread_matrix(rng, 17, 5, spread=12)
    exact = O.exact_matmul(A, B)
    em = O.emulated_matmul(A, B, s)
    bound = O.emulation_error_bound(A, B, s) + np.spacing(np.abs(exact))
    err = np.abs(em - exact)
    assert np.all(err <= bound)
    if s <= 4:   # the emulation really truncates (the bound is not vacuous)
        assert err.max() > 1e-6 * bound.max()


def test_emulated_exchange_converges_to_fp64(small):
    _, B, C, _ = small
    K = O.exchange(B, C)
    scale = np.max(np.abs(K))
    errs = {s: np.max(np.abs(O.emulated_exchange(B, C, s) - K)) / scale for s in (3, 5, 8)}
    assert errs[3] > errs[5] > errs[8]
    assert errs[3] < 1e-5 and errs[5] < 1e-10 and errs[8] < 1e-14


def test_emulated_exchange_per_block_counts(small):
    _, B, C, _ = small
    K_all8 = O.emulated_exchange(B, C, 8)
    K_mixed = O.emulated_exchange(B, C, [8, 3, 8])
    K = O.exchange(B, C)
    assert np.max(np.abs(K_mixed - K)) > 10 * np.max(np.abs(K_all8 - K))


# --- Table 1 and the adaptive rule -------------------------------------------------------

def _table1():
    rows = []
    for line in open(os.path.join(GOLDEN, "table1.txt")):
        if line.strip() and not line.startswith("#"):
            lo, lv, m, acc, sp = line.split()
            rows.append((float(lo), int(lv), None if m == "-" else int(m), float(acc), int(sp)))
    return rows


def test_table1_golden_values():
    rows = _table1()
    assert [(r[0], r[1], r[2], r[4]) for r in rows] == [(r[0], r[1], r[2], r[4]) for r in O.TABLE1]
    for lo, level, m, acc, splits in rows:
        assert O.slices_for_level(level) == splits
        if m is not None:
            assert O.slices_for_mantissa(m) == splits          # s = ceil((m+1)/8)
            assert abs(2.0 ** -m - acc) / acc < 0.05            # printed accuracy is 2^-m
        else:
            assert abs(2.0 ** -52 - acc) / acc < 0.05


def test_level_rule_boundaries():
    rows = _table1()
    for lo, level, _, _, _ in rows:
        if lo > 0:
            assert O.level_for(lo) == level                      # lower bound is inclusive
            assert O.level_for(lo * (1 - 1e-12)) == level - 1    # just below goes one level down
    assert O.level_for(1.0) == 4 and O.level_for(0.0) == 0


def test_level_schedule_monotone_and_starts_low():
    E = [-100.0, -100.5, -100.5001, -100.4, -100.50010001, -100.500100010001, -100.500100010001]
    lv = O.level_schedule(E)
    assert lv[0] == lv[1] == 4
    assert all(a >= b for a, b in zip(lv, lv[1:]))
    # a big jump after precision rose does not lower precision again
    assert lv[4] <= lv[3]
    assert lv[-1] == 0


def test_flop_model():
    for nscr, nbf, naux, nocc in [(10000, 100, 300, 20), (360000, 600, 1800, 120), (5000, 100, 300, 20)]:
        assert O.flops_J(nscr, naux) == 2 * nscr * naux + 2 * nscr * naux
        assert O.flops_K(nscr, nbf, naux, nocc) == 2 * nscr * naux * nocc + 2 * nbf * nbf * naux * nocc
        # K needs at least N_occ times the FLOPs of J because N_scr <= N_bf^2
        assert O.flops_K(nscr, nbf, naux, nocc) >= nocc * O.flops_J(nscr, naux)


def test_df_tensor_rows_is_the_leading_block(small):
    """Rows of B depend only on the leading auxiliary functions (forward substitution);
    two triangular solves agree within n u cond(L) |B|."""
    mol, B, _, _ = small
    Bk = inputs.df_tensor_rows(mol, 128)
    V = inputs.metric(mol)
    tol = V.shape[0] * 2.0 ** -52 * math.sqrt(np.linalg.cond(V)) * np.max(np.abs(B))
    assert np.max(np.abs(Bk - B[:128])) <= tol


# --- Schwarz screening (Section 2.1) ---------------------------------------------

def test_schwarz_self_coulomb_is_the_four_index_diagonal(tiny):
    mol = tiny[0]
    eri = O.eri4(mol.ao_xyz, mol.ao_exp)
    n = mol.nao
    diag = np.array([[eri[a, b, a, b] for b in range(n)] for a in range(n)])
    assert np.allclose(O.pair_self_coulomb(mol.ao_xyz, mol.ao_exp), diag, rtol=1e-13, atol=0)


def test_schwarz_inequality_bounds_the_integrals(tiny):
    """The Cauchy-Schwarz bounds behind the screening: |(ab|cd)| <= sqrt((ab|ab)(cd|cd)) and
    |(P|ab)| <= sqrt((P|P)(ab|ab)), brute force over every index."""
    mol, T, V = tiny[0], tiny[1], tiny[2]
    eri = O.eri4(mol.ao_xyz, mol.ao_exp)
    q = np.sqrt(O.pair_self_coulomb(mol.ao_xyz, mol.ao_exp))
    assert np.all(np.abs(eri) <= q[:, :, None, None] * q[None, None, :, :] * (1 + 1e-12))
    assert np.all(np.abs(T) <= np.sqrt(np.diag(V))[:, None, None] * q[None, :, :] * (1 + 1e-12))


def test_schwarz_mask_of_the_generator_and_the_zeros_of_B():
    """The input generator's screening equals the oracle's on a 30-atom chain, keeps every
    diagonal pair, and the screened pairs are exact zeros in every B_P."""
    mol = inputs.chain_molecule(30, 5)
    keep = O.schwarz_keep(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp, 1e-12)
    assert np.array_equal(inputs.schwarz_pairs(mol, 1e-12), keep)
    assert keep.all(axis=None) is not True and np.all(np.diag(keep)) and 0.2 < keep.mean() < 0.6
    B = inputs.df_tensor(mol, 1e-12)
    assert np.all(B[:, ~keep] == 0.0) and np.all(np.abs(B).max(axis=0)[keep] > 0.0)
