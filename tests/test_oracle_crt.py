"""Pins of the CRT (Ozaki scheme II) emulation oracle."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import crt_oracle as CO
from oracle import df_oracle as O


def test_moduli_are_greedy_pairwise_coprime():
    mods = CO.moduli(CO.MAX_MODULI)
    assert mods[:6] == [256, 255, 253, 251, 247, 241]
    assert all(a > b for a, b in zip(mods, mods[1:]))
    for i in range(len(mods)):
        for j in range(i):
            assert math.gcd(mods[i], mods[j]) == 1
    # every integer skipped between two taken ones shares a factor with an earlier one
    for m in range(mods[-1] + 1, 257):
        if m not in mods:
            assert any(math.gcd(m, t) > 1 for t in mods if t > m)
    assert CO.modulus_product(16) < 2 ** 128        # four 32-bit limbs hold M


@pytest.mark.parametrize("K", [1, 64, 1000, 1200, 32000])
def test_operand_width_is_the_largest_that_fits(K):
    for n in range(3, CO.MAX_MODULI + 1):
        q = CO.operand_bits(K, n)
        Mn = CO.modulus_product(n)
        assert 2 <= q <= 63
        assert K * 2 ** (2 * q - 1) < Mn
        assert q == 63 or K * 2 ** (2 * q + 1) >= Mn


def test_moduli_for_table1_levels():
    # 1200-term sums (the first exchange GEMM of the 240-atom molecule)
    got = {m: CO.moduli_for_bits(1200, m) for m in (23, 31, 39, 47, 52)}
    for m, n in got.items():
        assert CO.operand_bits(1200, n) >= m + 1 > CO.operand_bits(1200, n - 1)
    assert got[23] < got[31] < got[39] < got[47] <= got[52]


def test_residues_range_and_congruence():
    rng = np.random.default_rng(0)
    Ai = rng.integers(-2 ** 62, 2 ** 62, size=(7, 9), dtype=np.int64)
    for m in CO.moduli(16):
        r = CO.residues(Ai, m)
        assert r.min() >= -((m - 1) // 2) and r.max() <= m // 2
        assert np.all(np.mod(Ai - r, m) == 0)


@pytest.mark.parametrize("n", [4, 8, 12, 16])
def test_residue_path_equals_exact_integer_product(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((5, 11)) * np.exp(rng.uniform(-6, 6, (5, 1)))
    B = rng.standard_normal((4, 11))
    B[1] = 0.0                                              # a zero row
    K = A.shape[1]
    q = CO.operand_bits(K, n)
    mods = CO.moduli(n)
    _, Ai = CO.scaled_integers(A, q)
    _, Bi = CO.scaled_integers(B, q)
    P = CO.crt_reconstruct(CO.residue_products(Ai, Bi, mods), mods)
    for r in range(5):
        for c in range(4):
            exact = sum(int(Ai[r, k]) * int(Bi[c, k]) for k in range(K))
            assert P[r, c] == exact
    assert all(P[r, 1] == 0 for r in range(5))


def test_integer_matrices_multiply_exactly():
    rng = np.random.default_rng(3)
    A = rng.integers(-100, 101, (6, 40)).astype(np.float64) * 2.0 ** 5
    B = rng.integers(-100, 101, (7, 40)).astype(np.float64) * 2.0 ** -3
    assert np.array_equal(CO.emulated_gemm_crt(A, B, 6), A @ B.T)


@pytest.mark.parametrize("n", [5, 9, 13])
def test_error_within_bound_against_exact_products(n):
    rng = np.random.default_rng(10 + n)
    A = rng.standard_normal((4, 24)) * np.exp(rng.uniform(-4, 4, (4, 1)))
    B = rng.standard_normal((3, 24))
    out = CO.emulated_gemm_crt(A, B, n)
    ex = np.empty_like(out)
    for r in range(4):
        for c in range(3):
            ex[r, c] = float(sum(Fraction(float(A[r, k])) * Fraction(float(B[c, k])) for k in range(24)))
    bound = CO.error_bound(A, B, n) + np.spacing(np.abs(ex))
    assert np.all(np.abs(out - ex) <= bound)


def test_more_moduli_do_not_do_worse():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((6, 50))
    B = rng.standard_normal((5, 50))
    ref = A @ B.T
    errs = [np.max(np.abs(CO.emulated_gemm_crt(A, B, n) - ref)) for n in (4, 6, 8, 10, 12)]
    assert all(a >= b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-12 * np.max(np.abs(ref))


def test_agrees_with_slices_at_matching_width():
    # q = 8s: the CRT width that resolves x like s slices; both errors are of one size
    rng = np.random.default_rng(11)
    A = rng.standard_normal((8, 64))
    B = rng.standard_normal((8, 64))
    ref = A @ B.T
    for s in (3, 4, 5):
        n = CO.moduli_for_bits(64, 8 * s - 1)
        e_crt = np.max(np.abs(CO.emulated_gemm_crt(A, B, n) - ref))
        e_sl = np.max(np.abs(O.emulated_matmul(A, B.T, s) - ref))
        assert e_crt <= 4 * e_sl


def test_transpose_and_power_of_two_scaling_are_exact():
    # the procedure treats rows of A and rows of B alike, and a power-of-two
    # scale only moves the row exponent
    rng = np.random.default_rng(21)
    A = rng.standard_normal((5, 30)) * np.exp(rng.uniform(-3, 3, (5, 1)))
    B = rng.standard_normal((4, 30))
    out = CO.emulated_gemm_crt(A, B, 9)
    assert np.array_equal(CO.emulated_gemm_crt(B, A, 9), out.T)
    assert np.array_equal(CO.emulated_gemm_crt(A * 2.0 ** 37, B * 2.0 ** -11, 9), out * 2.0 ** 26)
