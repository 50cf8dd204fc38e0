"""CPU oracle for the adaptive-precision density-fitting J/K build.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never calls it and shares no code with it.

Plain, slow, obviously correct NumPy in FP64.  Each function cites the part
of the paper it restates (arXiv 2601.08077, "Accelerating Density Fitting
with Adaptive-precision and 8-bit Integer on AI Accelerators"):

* Section 2.1, Eq. df / Eq. cderi: DF tensor B = L^{-1}(P|mu nu), L L^T = (P|Q).
* Section 2.1, Eqs. df-j-1/df-j-2: rho_P = sum B_Pmn D_mn, J_mn = sum_P B_Pmn rho_P.
* Section 2.1, Eqs. df-k-1/df-k-2: X_Pmi = sum_n B_Pmn C_ni, K_mn = sum_Pi X_Pmi X_Pni.
* Section 3.3, Eqs. df-k-blk-1/2: K accumulated over blocks of auxiliary functions.
* Section 3.2: FP64 GEMM emulated by s INT8 slices, s = ceil((m+1)/8).
* Section 3.2, Table 1: energy-change rule for the emulation level; no
  return to a lower precision once a higher one was used.
* Section 3.1: FLOP model of the J and K builds.

The slice emulation follows the fixed-point reading of Section 3.2 (the paper
delegates the details to the library it calls): per-row and per-column
power-of-two exponents, balanced signed 8-bit digits, exact integer products
of slice pairs whose digit indices sum to less than s, and a single rounding
of the exactly recombined sum to FP64.

Parity pins (tests/test_oracle_pins.py): closed-form Gaussian integrals, the
Boys function limits, symmetry and positive definiteness of the metric, the
aux-normalisation invariance of B, J = J^T, K = K^T >= 0, E_J and E_K computed
two ways, a quadruple-loop K from the four-index DF integrals, the variational
bound E_J(DF) <= E_J(exact), exact digit reconstruction, exact emulation of
integer-valued matrices, the emulation error bound against exact rational
products, Table 1's printed values and the rule's boundaries and monotonicity.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

PI = math.pi

# ---------------------------------------------------------------------------
# Integrals over normalised s-type Gaussians (inputs of Eq. df / Eq. cderi)
# ---------------------------------------------------------------------------


def boys_f0(T):
    """F0(T) = int_0^1 exp(-T u^2) du = sqrt(pi/T) erf(sqrt T) / 2."""
    from scipy.special import erf
    T = np.asarray(T, dtype=np.float64)
    out = np.empty_like(T)
    small = T < 1e-10
    out[small] = 1.0 - T[small] / 3.0 + T[small] ** 2 / 10.0
    t = T[~small]
    out[~small] = 0.5 * np.sqrt(PI / t) * erf(np.sqrt(t))
    return out


def norm_s(a):
    return (2.0 * np.asarray(a, dtype=np.float64) / PI) ** 0.75


def gaussian_product(a, A, b, B):
    """p = a+b, P = (aA+bB)/p, K_ab = exp(-ab/p |A-B|^2) (broadcasting)."""
    p = a + b
    K = np.exp(-a * b / p * np.sum((A - B) ** 2, axis=-1))
    P = (a[..., None] * A + b[..., None] * B) / p[..., None]
    return p, P, K


def coulomb_ss(p, P, q, Q):
    """(unit-weight s Gaussian exp(-p|r-P|^2) | exp(-q|r-Q|^2)) = 2pi^{5/2}/(pq sqrt(p+q)) F0(.)."""
    R2 = np.sum((P - Q) ** 2, axis=-1)
    return 2.0 * PI ** 2.5 / (p * q * np.sqrt(p + q)) * boys_f0(p * q / (p + q) * R2)


def metric(aux_xyz, aux_exp):
    """(P|Q) over normalised auxiliary s primitives."""
    g = aux_exp
    V = coulomb_ss(g[:, None], aux_xyz[:, None, :], g[None, :], aux_xyz[None, :, :])
    return norm_s(g)[:, None] * norm_s(g)[None, :] * V


def int3c(ao_xyz, ao_exp, aux_xyz, aux_exp):
    """(P|mu nu) over normalised primitives, shape [naux, nao, nao]."""
    a = ao_exp
    p, Pc, Kab = gaussian_product(a[:, None], ao_xyz[:, None, :], a[None, :], ao_xyz[None, :, :])
    nab = norm_s(a)[:, None] * norm_s(a)[None, :] * Kab
    out = np.empty((len(aux_exp), len(a), len(a)))
    for P in range(len(aux_exp)):
        g = np.full_like(p, aux_exp[P])
        out[P] = norm_s(aux_exp[P]) * nab * coulomb_ss(g, aux_xyz[P][None, None, :], p, Pc)
    return out


def eri4(ao_xyz, ao_exp):
    """Exact four-centre (ab|cd) over normalised s primitives (tiny nao only)."""
    a = ao_exp
    p, Pc, Kab = gaussian_product(a[:, None], ao_xyz[:, None, :], a[None, :], ao_xyz[None, :, :])
    nab = norm_s(a)[:, None] * norm_s(a)[None, :] * Kab
    n = len(a)
    return (nab[:, :, None, None] * nab[None, None, :, :] *
            coulomb_ss(p[:, :, None, None], Pc[:, :, None, None, :],
                       p[None, None, :, :], Pc[None, None, :, :, :])).reshape(n, n, n, n)


def pair_self_coulomb(ao_xyz, ao_exp):
    """(ab|ab) for every AO pair: the Coulomb self-interaction of the normalised
    Gaussian product a*b (Gaussian product theorem, then the s-type Coulomb
    integral at zero separation)."""
    a = ao_exp
    p, Pc, Kab = gaussian_product(a[:, None], ao_xyz[:, None, :], a[None, :], ao_xyz[None, :, :])
    nab = norm_s(a)[:, None] * norm_s(a)[None, :] * Kab
    return nab * nab * coulomb_ss(p, Pc, p, Pc)


def schwarz_keep(ao_xyz, ao_exp, aux_xyz, aux_exp, tau):
    """Schwarz screening of Section 2.1: keep the pair (a, b) unless
    sqrt((ab|ab) max_P (P|P)) < tau.  Returns a bool [nao, nao]."""
    pp = float(np.max(np.diag(metric(aux_xyz, aux_exp))))
    return np.sqrt(pair_self_coulomb(ao_xyz, ao_exp) * pp) >= tau


# ---------------------------------------------------------------------------
# DF tensor, Section 2.1 Eq. cderi
# ---------------------------------------------------------------------------


def cholesky(V):
    """Lower Cholesky factor by the column algorithm; raises if not PD."""
    n = V.shape[0]
    L = np.zeros_like(V)
    for j in range(n):
        d = V[j, j] - np.dot(L[j, :j], L[j, :j])
        if not d > 0.0:
            raise np.linalg.LinAlgError("metric not positive definite at column %d" % j)
        L[j, j] = math.sqrt(d)
        L[j + 1:, j] = (V[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def forward_substitution(L, T):
    """Solve L Y = T row by row (T: [n, m])."""
    Y = np.empty_like(T)
    for i in range(L.shape[0]):
        Y[i] = (T[i] - L[i, :i] @ Y[:i]) / L[i, i]
    return Y


def df_tensor(int3c_, metric_):
    """B^q_mn = sum_p (mn|p) L^{-1}_pq with L L^T = (P|Q) (Eq. cderi)."""
    naux, nao, _ = int3c_.shape
    L = cholesky(metric_)
    return forward_substitution(L, int3c_.reshape(naux, -1)).reshape(naux, nao, nao)


# ---------------------------------------------------------------------------
# Coulomb and exchange builds, Section 2.1 Eqs. df-j-1 .. df-k-2
# ---------------------------------------------------------------------------


def rho(B, D):
    """Y^q = sum_ij B^q_ij D_ij (Eq. df-j-1)."""
    return np.einsum("pmn,mn->p", B, D)


def coulomb(B, rho_):
    """J_ij = sum_q B^q_ij Y^q (Eq. df-j-2)."""
    return np.einsum("pmn,p->mn", B, rho_)


def exchange_X(B, C):
    """W^q_is = sum_r B^q_ir C_rs (Eq. df-k-1), shape [naux, nao, nocc]."""
    return B @ C


def exchange(B, C):
    """K_ij = sum_q sum_s W^q_is W^q_js (Eq. df-k-2)."""
    X = exchange_X(B, C)
    naux, nao, nocc = X.shape
    Xt = X.transpose(1, 0, 2).reshape(nao, naux * nocc)
    return Xt @ Xt.T


def energies(D, J, K):
    """E_J = 1/2 tr(D J), E_K = -1/2 tr(D K) (K with occupations not folded in)."""
    return 0.5 * float(np.sum(D * J)), -0.5 * float(np.sum(D * K))


def energies_alt(B, C, rho_):
    """Second route: E_J = 1/2 rho.rho, E_K = -sum_P ||C^T B_P C||_F^2."""
    EJ = 0.5 * float(rho_ @ rho_)
    M = np.einsum("ni,pnm,mj->pij", C, B, C)
    return EJ, -float(np.sum(M * M))


def exchange_bruteforce(B, D):
    """K_full[a,b] = sum_cd (ac|bd)_DF D_cd with (ab|cd)_DF = sum_P B_Pab B_Pcd.

    A quadruple loop over the four-index DF integrals (tiny nao only); the X
    route gives K = K_full / 2 because D = 2 C C^T.
    """
    naux, n, _ = B.shape
    eri = np.einsum("pab,pcd->abcd", B, B)
    K = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            s = 0.0
            for c in range(n):
                for d in range(n):
                    s += eri[a, c, b, d] * D[c, d]
            K[a, b] = s
    return K


# ---------------------------------------------------------------------------
# INT8 slice emulation of an FP64 GEMM, Section 3.2
# ---------------------------------------------------------------------------

S_MAX = 8          # digits kept per value: 8 x 8 bits = 64 >= 63 bits of RNE(x 2^63)
HEADROOM = 127.0 / 128.0


def row_exponents(A):
    """Smallest e per row with max_k |A_rk| < (127/128) 2^e; zero rows get 0."""
    A = np.asarray(A, dtype=np.float64)
    amax = np.max(np.abs(A), axis=1) if A.shape[1] else np.zeros(A.shape[0])
    e = np.zeros(A.shape[0], dtype=np.int64)
    nz = amax > 0
    m, E = np.frexp(amax[nz])              # amax = m 2^E, m in [0.5, 1)
    # amax < 127/128 2^e  <=>  e = E if m < 127/128 else E+1
    e[nz] = E + (m >= HEADROOM)
    return e


def split_rows(A, s=S_MAX):
    """Balanced signed 8-bit digits of each row (Section 3.2).

    x = A_rk 2^{-e_r} (exact); N = RNE(x 2^63) as int64; then seven times
    d_low = ((N & 0xFF) ^ 0x80) - 128, N = (N - d_low) >> 8, and the rest is
    the top digit, so x 2^63 = sum_t d_t 256^{7-t} with every d_t in
    [-128, 127] and |d_0| <= 127.  Returns (e [rows], digits [s, rows, cols]
    int8), digits t = 0..s-1 most significant first.
    """
    A = np.asarray(A, dtype=np.float64)
    e = row_exponents(A)
    x = np.ldexp(A, -e[:, None])
    N = np.rint(np.ldexp(x, 63)).astype(np.int64)   # |x| < 1 so |N| < 2^63
    digits = np.empty((S_MAX,) + A.shape, dtype=np.int64)
    for t in range(S_MAX - 1, 0, -1):
        d = ((N & 0xFF) ^ 0x80) - 128
        digits[t] = d
        N = (N - d) >> 8
    digits[0] = N
    return e, digits[:s].astype(np.int8)


def reconstruct(e, digits):
    """Exact value sum_t d_t 2^{e_r - 7 - 8t} of the digits given, rounded once to FP64."""
    s = digits.shape[0]
    R = np.zeros(digits.shape[1:], dtype=object)
    for t in range(s):
        R = R * 256 + digits[t].astype(np.int64).astype(object)
    k = np.broadcast_to(np.asarray(e)[:, None], digits.shape[1:]) - 7 - 8 * (s - 1)
    return _ldexp_exact_array(R, k)


def slice_products(Ad, Bd, s):
    """S_g = sum_{t+u=g} A_t B_u^T for g < s: exact int64 [s, M, N] (Section 3.2).

    Ad: [>=s, M, K] digits of A's rows; Bd: [>=s, N, K] digits of B's columns.
    """
    Ad = Ad.astype(np.int64)
    Bd = Bd.astype(np.int64)
    M, N = Ad.shape[1], Bd.shape[1]
    S = np.zeros((s, M, N), dtype=np.int64)
    for g in range(s):
        for t in range(g + 1):
            S[g] += Ad[t] @ Bd[g - t].T
    return S


def recombine(S, ea, eb):
    """fl64( 2^{ea_r + eb_c - 14} sum_g 2^{-8g} S_g ), rounded once (Section 3.2)."""
    s = S.shape[0]
    R = np.zeros(S.shape[1:], dtype=object)
    for g in range(s):
        R = R + (S[g].astype(object) << (8 * (s - 1 - g)))
    k = (np.asarray(ea, dtype=np.int64)[:, None] + np.asarray(eb, dtype=np.int64)[None, :]
         - (14 + 8 * (s - 1)))
    return _ldexp_exact_array(R, k)


def _ldexp_exact_array(R, k):
    """Correctly rounded FP64 of R 2^k for Python-int R (no subnormal results)."""
    flat = np.array([float(r) for r in np.asarray(R, dtype=object).ravel()])
    return np.ldexp(flat, np.asarray(k, dtype=np.int64).ravel()).reshape(np.shape(R))


def emulated_matmul(A, B, s):
    """A @ B emulated with s INT8 slices per operand (rows of A, columns of B)."""
    ea, Ad = split_rows(A, s)
    eb, Bd = split_rows(np.ascontiguousarray(np.asarray(B).T), s)
    return recombine(slice_products(Ad, Bd, s), ea, eb)


def emulated_exchange(B, C, s, block=128, return_parts=False):
    """K of Eq. df-k-2 with both contractions emulated at s slices.

    Eq. df-k-blk-1: X = B C with one exponent per (P, mu) row of B and one per
    column of C.  Eq. df-k-blk-2: per block of `block` auxiliary functions,
    X_blk [mu, (P, i)] gets one exponent per (block, mu) row and K_blk =
    X_blk X_blk^T is emulated; K is the FP64 sum of the blocks in block order.
    `s` may be an int or a per-block list (the first GEMM of a block uses that
    block's count too).
    """
    naux, nao, _ = B.shape
    nocc = C.shape[1]
    nblk = (naux + block - 1) // block
    s_blk = [s] * nblk if np.isscalar(s) else list(s)
    X = np.empty((naux, nao, nocc))
    K = np.zeros((nao, nao))
    parts = []
    for b in range(nblk):
        p0, p1 = b * block, min((b + 1) * block, naux)
        sb = int(s_blk[b])
        Xb = emulated_matmul(B[p0:p1].reshape(-1, nao), C, sb).reshape(p1 - p0, nao, nocc)
        X[p0:p1] = Xb
        Xt = Xb.transpose(1, 0, 2).reshape(nao, -1)
        Kb = emulated_matmul(Xt, Xt.T, sb)
        parts.append(Kb)
        K += Kb
    if return_parts:
        return K, X, parts
    return K


def emulation_error_bound(A, B, s):
    """Elementwise bound on |emulated_matmul(A,B,s) - A@B| (exact arithmetic).

    Each value is x = sum_{t<8} d_t 2^{-7-8t} + r with |r| <= 2^-64 (rounding
    of x 2^63); dropping pairs with t+u >= s loses at most
    sum_{g>=s} (g+1) 2^{14} 2^{-14-8g} <= 1.01 (s+1) 2^{-8s} per product, the
    rounding terms at most 2^-63; the final rounding adds half an ulp.
    """
    K = A.shape[1]
    ea = row_exponents(A)
    eb = row_exponents(np.asarray(B).T)
    scale = np.ldexp(1.0, (ea[:, None] + eb[None, :]).astype(np.int64))
    per = 1.01 * (s + 1) * 2.0 ** (-8 * s) + 2.0 ** -63
    return K * scale * per


def exact_matmul(A, B):
    """Exact rational A @ B, rounded once to FP64 (tiny shapes only)."""
    M, K = A.shape
    N = B.shape[1]
    out = np.empty((M, N))
    Af = [[Fraction(float(v)) for v in row] for row in A]
    Bf = [[Fraction(float(B[k, n])) for n in range(N)] for k in range(K)]
    for m in range(M):
        for n in range(N):
            out[m, n] = float(sum(Af[m][k] * Bf[k][n] for k in range(K)))
    return out


# ---------------------------------------------------------------------------
# Adaptive precision selection, Section 3.2 and Table 1
# ---------------------------------------------------------------------------

# (lower bound of Delta E_rel, level, m_emu, accuracy printed, INT8 splits)
TABLE1 = (
    (2e-6, 4, 23, 1.2e-7, 3),
    (5e-9, 3, 31, 4.7e-10, 4),
    (2e-11, 2, 39, 1.8e-12, 5),
    (7e-14, 1, 47, 7.1e-15, 6),
    (0.0, 0, None, 2.2e-16, 0),
)
START_LEVEL = 4


def slices_for_mantissa(m):
    """s_emu = ceil((m_emu + 1) / 8) (Section 3.2)."""
    return -(-(m + 1) // 8)


def level_for(dE_rel):
    """Table 1: the emulation level for the next iteration given Delta E_rel."""
    for lo, level, _, _, _ in TABLE1:
        if dE_rel >= lo:
            return level
    return 0


def slices_for_level(level):
    """INT8 splits for a level (0 means native FP64)."""
    for _, lv, m, _, _ in TABLE1:
        if lv == level:
            return 0 if m is None else slices_for_mantissa(m)
    raise ValueError(level)


def relative_change(E_prev, E_cur):
    """Delta E_rel_i = |(E_i - E_{i-1}) / E_i|."""
    return abs((E_cur - E_prev) / E_cur)


def level_schedule(energies_):
    """Levels used by iterations 0..n given the energies E_0..E_{n-1} seen so far.

    Iterations 0 and 1 run at the start level (no energy change exists before
    the second energy); afterwards level_{k+1} = min(level_k, rule(dE_rel_k)):
    the level never returns to a lower precision (Section 3.2).
    """
    levels = [START_LEVEL]
    for k in range(len(energies_)):
        if k == 0:
            levels.append(levels[-1])
            continue
        dE = relative_change(energies_[k - 1], energies_[k])
        levels.append(min(levels[-1], level_for(dE)))
    return levels


# ---------------------------------------------------------------------------
# FLOP model, Section 3.1
# ---------------------------------------------------------------------------


def flops_J(n_scr, n_aux):
    return 4 * n_scr * n_aux


def flops_K(n_scr, n_bf, n_aux, n_occ):
    return 2 * (n_scr + n_bf * n_bf) * n_aux * n_occ
