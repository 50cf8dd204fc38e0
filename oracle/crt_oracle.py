"""CPU oracle for the Chinese-remainder (CRT) variant of the emulated FP64 GEMM.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import it.  The CUDA library never calls it and
shares no code with it.

The paper builds K with an FP64 GEMM emulated by INT8 slices (Section 3.2) and
names, in Section 2.3, the other INT8 route: Ozaki scheme II (Ozaki, Uchino
and Imamura, 2025), which scales the FP64 operands to integers and multiplies
them exactly through their residues modulo several small coprime integers;
Section 4.5 reports that with such a library the emulation level had to be
guessed, because it takes a number of moduli, not an accuracy.  Here the
operand width follows from the moduli, so the level of Table 1 maps to a
modulus count exactly (`moduli_for_bits`).

The steps, for out = A B^T with A [M, K] and B [N, K]:

1. moduli m_1 > m_2 > ... : the integers <= 256 taken greedily downwards,
   each coprime to all taken before; M_n = m_1 ... m_n;
2. operand width q: the largest integer with K 2^(2q-1) < M_n (then every
   |sum_k A'_rk B'_ck| <= K 2^(2q-2) < M_n / 2), at most 63;
3. row exponents e (the smallest e with max|row| < (127/128) 2^e, 0 for a
   zero row) and integers A' = RNE(A 2^(q-1-e)) per row (and B' likewise);
4. residues a_i = A' mod m_i taken in [-floor((m_i-1)/2), floor(m_i/2)], so
   |a_i| <= 128 (exact in the BF16 digit carriers of the GPU);
5. per modulus an exact integer GEMM S_i = a_i b_i^T and y_i = S_i mod m_i;
6. the Chinese remainder theorem gives P' = sum_k A'B' as the unique integer
   in (-M_n/2, M_n/2] congruent to y_i modulo every m_i;
7. out = fl64(P' 2^(e_r + f_c - 2(q-1))), one rounding (to nearest even).

Pins (tests/test_oracle_crt.py): the moduli are pairwise coprime and greedy
(brute force); q is the largest width that fits; the residue path equals the
exact integer product of the scaled operands (plain Python integers, a route
without residues); integer-valued matrices multiply exactly; the error against
the exact rational product stays within K 2^(e_r+f_c-q+1) (1 + 2^-q) plus the
final half ulp; more moduli never do worse on a random case.
"""
from __future__ import annotations

import math

import numpy as np

from . import df_oracle as O

MAX_MODULI = 16
HEADROOM = 127.0 / 128.0


def moduli(n):
    """The first n moduli: greedy downwards from 256, pairwise coprime (step 1)."""
    out = []
    m = 256
    while len(out) < n and m >= 2:
        if all(math.gcd(m, t) == 1 for t in out):
            out.append(m)
        m -= 1
    if len(out) < n:
        raise ValueError("not enough moduli")
    return out


def modulus_product(n):
    return math.prod(moduli(n))


def operand_bits(K, n):
    """Largest q <= 63 with K 2^(2q-1) < M_n (step 2); 0 if none >= 2 fits."""
    Mn = modulus_product(n)
    q = 0
    for c in range(2, 64):
        if K * (1 << (2 * c - 1)) < Mn:
            q = c
    return q


def moduli_for_bits(K, bits):
    """Fewest moduli whose width q reaches `bits` + 1 (the slice scheme's
    s = (m + 1)/8 slices resolve x to 2^(e - 8s); the width q resolves it to
    2^(e - q), so level m of Table 1 needs q >= m + 1)."""
    for n in range(2, MAX_MODULI + 1):
        if operand_bits(K, n) >= bits + 1:
            return n
    return 0


def scaled_integers(A, q):
    """(e, A') with A' = RNE(A 2^(q-1-e)) per row, int64 (step 3)."""
    A = np.asarray(A, dtype=np.float64)
    e = O.row_exponents(A)
    x = np.ldexp(A, -e[:, None])                      # exact, |x| < 127/128
    Ai = np.rint(np.ldexp(x, q - 1)).astype(np.int64)  # |A'| < 2^(q-1)
    return e, Ai


def residues(Ai, m):
    """A' mod m in [-floor((m-1)/2), floor(m/2)] (step 4)."""
    r = np.mod(Ai, m)                 # [0, m)
    return np.where(r > m // 2, r - m, r)


def residue_products(Ai, Bi, mods):
    """y_i = (a_i b_i^T) mod m_i, uint8 [n, M, N] (step 5)."""
    Y = np.empty((len(mods), Ai.shape[0], Bi.shape[0]), dtype=np.uint8)
    for i, m in enumerate(mods):
        S = residues(Ai, m) @ residues(Bi, m).T       # |S| <= K 2^14: exact int64
        Y[i] = np.mod(S, m)
    return Y


def crt_reconstruct(Y, mods):
    """The integer in (-M/2, M/2] with the residues Y (step 6), Python ints."""
    Mn = math.prod(mods)
    W = []
    for m in mods:
        c = Mn // m
        W.append(c * pow(c, -1, m))                   # = 1 mod m, = 0 mod the others
    out = np.empty(Y.shape[1:], dtype=object)
    for idx in np.ndindex(*Y.shape[1:]):
        x = sum(int(Y[(i,) + idx]) * W[i] for i in range(len(mods))) % Mn
        out[idx] = x - Mn if 2 * x > Mn else x
    return out


def emulated_gemm_crt(A, B, n):
    """out = A B^T (A [M, K], B [N, K]) emulated with n moduli (steps 1-7)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    K = A.shape[1]
    mods = moduli(n)
    q = operand_bits(K, n)
    if q < 2:
        raise ValueError("too few moduli for K")
    ea, Ai = scaled_integers(A, q)
    eb, Bi = scaled_integers(B, q)
    P = crt_reconstruct(residue_products(Ai, Bi, mods), mods)
    k = ea[:, None] + eb[None, :] - 2 * (q - 1)
    return O._ldexp_exact_array(P, k)


def error_bound(A, B, n):
    """Elementwise bound on |emulated_gemm_crt(A, B, n) - A B^T| in exact
    arithmetic, before the final rounding: A = (A' + da) 2^(e-q+1) with
    |da| <= 1/2 and |A'| <= 2^(q-1), so each product errs by at most
    2^(e+f-2q+2) (2^(q-1) + 1/4) and K of them by K 2^(e+f-q+1) (1 + 2^-q)."""
    K = np.asarray(A).shape[1]
    q = operand_bits(K, n)
    ea = O.row_exponents(A)
    eb = O.row_exponents(B)
    return K * np.ldexp(1.0, (ea[:, None] + eb[None, :] - q + 1).astype(np.int64)) * (1.0 + 2.0 ** -q)
