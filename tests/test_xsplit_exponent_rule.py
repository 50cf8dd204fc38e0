"""The exponent rule the X split takes from the first GEMM's bound, against the oracle.

The first exchange GEMM hands the X split each row's exact int64 sums R with
scales k (X = fl64(R 2^k), the emulated product's one rounding) and, per row,
the bound g = max(bitlen(|R|) + k) over its nonzero sums.  The X split then
decides the row exponent without rounding every element: it is g + 1 exactly
when some element with bitlen(|R|) + k = g has a normalised 64-bit mantissa
u 2^(64 - bitlen) >= 127 2^57 - 2^10, else g.  This CPU test checks that
rule against the oracle's definition of the row exponent (the smallest e with
max |X| < 127/128 2^e, computed from the correctly rounded FP64 values) on
rows built around the threshold, where a wrong constant or a wrong tie rule
would show.  No GPU.
"""
import math

import numpy as np

from oracle import df_oracle as O

TOP_M = 0xFDFFFFFFFFFFFC00  # 127 2^57 - 2^10


def rule_exponent(Rs, ks):
    g = max(abs(R).bit_length() + k for R, k in zip(Rs, ks) if R != 0)
    hit = any(R != 0 and abs(R).bit_length() + k == g and (abs(R) << (64 - abs(R).bit_length())) >= TOP_M
              for R, k in zip(Rs, ks))
    return g + 1 if hit else g


def oracle_exponent(Rs, ks):
    # Python's int -> float conversion rounds to nearest even; ldexp by k is exact here
    X = np.array([[math.ldexp(float(R), k) for R, k in zip(Rs, ks)]])
    return int(O.row_exponents(X)[0])


def test_rule_matches_the_oracle_near_the_threshold():
    rng = np.random.default_rng(2024)
    checked = 0
    for _ in range(20000):
        cnt = int(rng.integers(1, 6))
        Rs, ks = [], []
        for _ in range(cnt):
            nb = int(rng.integers(8, 64))
            mode = rng.random()
            if mode < 0.6:
                # within a few units of the last kept bit of 127/128 of the binade
                d = 2 ** max(0, nb - 53)
                R = (127 << (nb - 7)) + int(rng.integers(-3, 4)) * (d // 2 if d > 1 else 1)
            elif mode < 0.7:
                R = 2 ** nb - 1 - int(rng.integers(0, 2 ** max(0, nb - 54) + 1))
            else:
                R = int(rng.integers(2 ** (nb - 1), 2 ** nb - 1, dtype=np.uint64))
            R = max(1, min(R, 2 ** 63 - 1))
            Rs.append(-R if rng.random() < 0.5 else R)
            ks.append(int(rng.integers(-80, 20)))
        assert rule_exponent(Rs, ks) == oracle_exponent(Rs, ks), (Rs, ks)
        checked += 1
    assert checked == 20000


def test_rule_at_the_exact_edges():
    # one element per row, scale 0: the largest mantissa below the threshold, the threshold
    # itself (a tie at 53 bits that rounds to the even 127 2^46), and one above
    for nb in (54, 60, 63):
        base = 127 << (nb - 7)
        half = 1 << (nb - 54)
        below, tie, above = base - half - 1, base - half, base - half + 1
        assert oracle_exponent([below], [0]) == nb and rule_exponent([below], [0]) == nb
        assert oracle_exponent([tie], [0]) == nb + 1 and rule_exponent([tie], [0]) == nb + 1
        assert oracle_exponent([above], [0]) == nb + 1 and rule_exponent([above], [0]) == nb + 1
