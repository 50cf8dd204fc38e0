"""GPU parity of libdf against the CPU oracle, through the C ABI.

Integer work (digits, exponents, slice-pair products) must be bit-exact.
FP64 results must be bit-exact where the fixed-point recombination is exact
(truncation T = 0), and otherwise within the bound of the dropped bits; the
J/K builds must meet the target tolerances max|dK| <= 1e-10 max|K| and
|dE| <= 1e-9 Eh at the full slice count.
"""
import math

import numpy as np
import pytest
import torch

from oracle import df_oracle as O
from paper_2601_08077_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def df():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_08077_gb300 import build, df as dfmod
    build.build_all()
    return dfmod


@pytest.fixture(scope="module")
def small():
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    return B, C, D


@pytest.fixture(scope="module")
def medium():
    mol, B, C, D = inputs.make_inputs(inputs.MEDIUM)
    return B, C, D


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def spread(rng, m, n, spread=20):
    return rng.standard_normal((m, n)) * np.exp2(rng.integers(-spread, 1, size=(m, n)))


def shift_T(s, k):
    """Truncation of the int64 fixed-point sum (same rule as the library)."""
    bound = sum((g + 1) * k * 16384 * 2 ** (8 * (s - 1 - g)) for g in range(s))
    bits = 0
    while 2 ** bits < bound:
        bits += 1
    return max(0, bits - 61)


def n_chunks(s, ktiles):
    return sum(-(-((g + 1) * ktiles) // 16) for g in range(s))


# --- split ------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(1, 1), (37, 53), (300, 1100), (129, 64)])
def test_split_bitexact(df, shape):
    rng = np.random.default_rng(sum(shape))
    A = spread(rng, *shape)
    A[0, : shape[1] // 2] = 0.0
    if shape[0] > 5:
        A[5] = 0.0
        A[3, 0] = 127 / 128 * 2.0 ** 7          # exactly on the headroom boundary
        A[4, -1] = -(2.0 ** -1070)              # subnormal
    e_ref, d_ref = O.split_rows(A, 8)
    e, d = df.split_int8(cuda(A), 8)
    assert np.array_equal(e.cpu().numpy(), e_ref.astype(np.int32))
    assert np.array_equal(d.cpu().numpy(), d_ref)


# --- slice-pair products -------------------------------------------------------------

@pytest.mark.parametrize("s", [1, 2, 3, 5, 8])
def test_slice_products_bitexact(df, s):
    rng = np.random.default_rng(100 + s)
    M, N, K = 300, 200, 1100      # 3 x 2 tiles with ragged edges; K > 1024 forces several chunks
    A = spread(rng, M, K, 10)
    B = spread(rng, N, K, 10)
    S, ea, eb = df.slice_products(cuda(A), cuda(B), s)
    ea_ref, Ad = O.split_rows(A, s)
    eb_ref, Bd = O.split_rows(B, s)
    S_ref = O.slice_products(Ad, Bd, s)
    assert np.array_equal(ea.cpu().numpy(), ea_ref.astype(np.int32))
    assert np.array_equal(eb.cpu().numpy(), eb_ref.astype(np.int32))
    assert np.array_equal(S.cpu().numpy(), S_ref)


def test_slice_products_at_the_exactness_limit(df):
    """Same-sign rows with near-full digits drive every 1024-product chunk to ~2^24."""
    K = 4096
    A = np.empty((130, K))
    A[:] = 0.9999999 * 0.992
    A[1::2] = -A[1::2]
    A[7] = 0.9921875 - 2.0 ** -40   # 127/128 - tiny: top digit 127, low digits near -128
    B = np.empty((140, K))
    B[:] = -(0.9921875 - 2.0 ** -45)
    s = 8
    S, _, _ = df.slice_products(cuda(A), cuda(B), s)
    ea, Ad = O.split_rows(A, s)
    eb, Bd = O.split_rows(B, s)
    S_ref = O.slice_products(Ad, Bd, s)
    per_chunk = np.abs(Ad[0].astype(np.int64)).max() * np.abs(Bd[0].astype(np.int64)).max() * 1024
    assert per_chunk > 2 ** 23          # the test really reaches the FP32 exactness limit
    assert np.array_equal(S.cpu().numpy(), S_ref)


# --- emulated product ----------------------------------------------------------------

@pytest.mark.parametrize("s", [1, 3, 4, 5, 6, 8])
def test_emulated_gemm_vs_oracle(df, s):
    rng = np.random.default_rng(200 + s)
    M, N, K = 150, 260, 700
    A = spread(rng, M, K, 14)
    B = spread(rng, N, K, 14)
    got = df.emulated_gemm(cuda(A), cuda(B), s).cpu().numpy()
    ref = O.emulated_matmul(A, B.T, s)
    ktiles = -(-K // 64)
    T = shift_T(s, ktiles * 64)
    if T == 0:
        assert np.array_equal(got, ref)
    else:
        ea, eb = O.row_exponents(A), O.row_exponents(B)
        unit = np.ldexp(1.0, (ea[:, None] + eb[None, :] - 14 - 8 * (s - 1) + T).astype(np.int64))
        bound = unit * (0.5 * n_chunks(s, ktiles) + 1) + 2 * np.spacing(np.abs(ref))
        assert np.all(np.abs(got - ref) <= bound)


# --- the DF builds --------------------------------------------------------------------------

def _ctx(df, B, nocc):
    naux, nao, _ = B.shape
    ctx = df.Context(nao, naux, nocc)
    Bt = cuda(B)
    ctx.setup(Bt)
    return ctx, Bt


@pytest.mark.parametrize("s", [3, 4, 5])
def test_exchange_small_bitexact_vs_oracle_emulation(df, small, s):
    B, C, D = small
    ctx, _ = _ctx(df, B, C.shape[1])
    K, st = ctx.build_K(cuda(C), s)
    ref = O.emulated_exchange(B, C, s)
    assert np.array_equal(K.cpu().numpy(), ref)
    assert st.nblk == 3 and list(st.slices[:3]) == [s] * 3


@pytest.mark.parametrize("s", [6, 7, 8])
def test_exchange_small_high_slices(df, small, s):
    B, C, D = small
    ctx, _ = _ctx(df, B, C.shape[1])
    K = ctx.build_K(cuda(C), s)[0].cpu().numpy()
    Kem = O.emulated_exchange(B, C, s)
    Kfp = O.exchange(B, C)
    scale = np.max(np.abs(Kfp))
    assert np.max(np.abs(K - Kem)) <= 1e-14 * scale
    assert np.max(np.abs(K - Kfp)) <= 1e-10 * scale
    assert np.array_equal(K, K.T)


def fp64_exchange_bound(B, C):
    """Two FP64 builds of K in different orders differ by at most twice the
    standard dot-product bound: gamma_n sum|terms| for X (n = nao) propagated
    into K, plus gamma_n sum|X||X| for K itself (n = naux nocc)."""
    u = 2.0 ** -53
    naux, nao, _ = B.shape
    nocc = C.shape[1]
    Xa = np.abs(B) @ np.abs(C)                      # bound on sum |B||C| per X element
    X = np.abs(B @ C)
    Xa_t = Xa.transpose(1, 0, 2).reshape(nao, -1)
    X_t = X.transpose(1, 0, 2).reshape(nao, -1)
    g1, g2 = 1.01 * nao * u, 1.01 * naux * nocc * u
    return 2 * (g1 * (Xa_t @ X_t.T + X_t @ Xa_t.T) + g2 * (X_t @ X_t.T)) + 1e-300


def test_exchange_native_fp64(df, small):
    B, C, D = small
    ctx, _ = _ctx(df, B, C.shape[1])
    K, st = ctx.build_K(cuda(C), 0)
    Kfp = O.exchange(B, C)
    assert st.fallback == 1
    assert np.all(np.abs(K.cpu().numpy() - Kfp) <= fp64_exchange_bound(B, C))


def test_exchange_per_block_slices(df, small):
    B, C, D = small
    ctx, _ = _ctx(df, B, C.shape[1])
    sl = [5, 3, 4]
    K, st = ctx.build_K_blocks(cuda(C), sl)
    assert list(st.slices[:3]) == sl
    assert np.array_equal(K.cpu().numpy(), O.emulated_exchange(B, C, sl))


def test_coulomb_and_energies(df, small):
    B, C, D = small
    ctx, _ = _ctx(df, B, C.shape[1])
    Dg = cuda(D)
    J, rho = ctx.build_J(Dg)
    K, _ = ctx.build_K(cuda(C), 8)
    r_ref = O.rho(B, D)
    J_ref = O.coulomb(B, r_ref)
    # FP64 sums in another order: |error| <= n u sum|terms| (n = nao^2 and naux terms)
    tol_r = 2 * B.shape[1] ** 2 * 2.0 ** -53 * np.abs(B).reshape(B.shape[0], -1) @ np.abs(D).ravel()
    assert np.all(np.abs(rho.cpu().numpy() - r_ref) <= tol_r + 1e-300)
    tol_J = 2 * B.shape[0] * 2.0 ** -53 * np.einsum("pmn,p->mn", np.abs(B), np.abs(r_ref)) + 1e-300
    assert np.all(np.abs(J.cpu().numpy() - J_ref) <= tol_J + np.einsum("pmn,p->mn", np.abs(B), tol_r))
    EJ, EJ2, EK = ctx.energy(Dg, J, K, rho)
    EJ_ref, EK_ref = O.energies(D, J_ref, O.exchange(B, C))
    assert abs(EJ - EJ_ref) <= 1e-9 and abs(EJ2 - EJ_ref) <= 1e-9 and abs(EK - EK_ref) <= 1e-9
    assert abs(EJ - EJ2) <= 1e-12 * abs(EJ)


def test_adaptive_controller_matches_rule(df, small):
    B, C, D = small
    ctx, _ = _ctx(df, B, C.shape[1])
    E = [-100.0, -100.5, -100.5001, -100.4, -100.50010001, -100.500100010001, -100.500100010001]
    levels = O.level_schedule(E)
    ctx.adaptive_reset()
    got = [4]
    for e in E:
        lv, ns = ctx.adaptive_next(e)
        got.append(lv)
        assert ns == O.slices_for_level(lv)
    assert got == levels
    for x in [1.0, 2e-6, 1.9999e-6, 5e-9, 4.9e-9, 2e-11, 1.9e-11, 7e-14, 6.9e-14, 0.0]:
        assert df.level_for(x) == O.level_for(x)


def test_adaptive_fp64_fallback_level(df, small):
    B, C, D = small
    ctx, _ = _ctx(df, B, C.shape[1])
    ctx.adaptive_reset(fp64_from_level=3)       # e.g. hardware where FP64 wins below level 4
    ctx.adaptive_next(-100.0)
    ctx.adaptive_next(-100.0000001)             # dE_rel ~ 1e-9 -> level 2
    lv, ns = ctx.adaptive_next(-100.00000011)
    assert lv <= 3 and ns == 0


def test_errors_are_reported(df, small):
    B, C, D = small
    ctx = df.Context(B.shape[1], B.shape[0], C.shape[1])
    with pytest.raises(df.DFError) as e:
        ctx.build_K(cuda(C), 3)                  # before setup
    assert e.value.status == -7
    ctx.setup(cuda(B))
    with pytest.raises(df.DFError) as e:
        ctx.build_K(cuda(C), 9)
    assert e.value.status == -1
    ctx.sync_status()


# --- the 120-atom molecule: the fixed-slice sweep ---------------------------------------------

def test_medium_sweep_against_fp64_oracle(df, medium):
    B, C, D = medium
    ctx, _ = _ctx(df, B, C.shape[1])
    Kfp = O.exchange(B, C)
    scale = np.max(np.abs(Kfp))
    Cg = cuda(C)
    errs = {}
    for s in range(3, 9):
        K = ctx.build_K(Cg, s)[0].cpu().numpy()
        errs[s] = np.max(np.abs(K - Kfp)) / scale
        assert np.array_equal(K, K.T)
    assert errs[3] > errs[4] > errs[5] > errs[6]
    assert errs[3] < 1e-5
    assert errs[5] <= 1e-10 and errs[8] <= 1e-10
    Kn = ctx.build_K(Cg, 0)[0].cpu().numpy()
    assert np.all(np.abs(Kn - Kfp) <= fp64_exchange_bound(B, C))
    Dg = cuda(D)
    J, rho = ctx.build_J(Dg)
    r_ref = O.rho(B, D)
    J_ref = O.coulomb(B, r_ref)
    assert np.max(np.abs(J.cpu().numpy() - J_ref)) <= 1e-12 * np.max(np.abs(J_ref))
    K8 = ctx.build_K(Cg, 8)[0]
    EJ, EJ2, EK = ctx.energy(Dg, J, K8, rho)
    EJ_ref, EK_ref = O.energies(D, J_ref, Kfp)
    assert abs(EJ - EJ_ref) <= 1e-9 and abs(EK - EK_ref) <= 1e-9


# --------------------------------------------------------------------------
# CTA-pair mode (DF_OPT_CLUSTER_PAIRS): two CTAs of a cluster run one
# M = 256 tcgen05 MMA over their two output tiles (cta_group::2), each
# staging its own A tile and half of the stacked B operand.  It must not
# change a bit.

def _random_df(seed, naux, nao, nocc):
    """A DF-shaped tensor (symmetric in mu, nu) and orbitals with row
    magnitudes spread over 2^-10..1, small enough for the exact oracle."""
    rng = np.random.default_rng(seed)
    B = spread(rng, naux * nao, nao, spread=10).reshape(naux, nao, nao)
    B = 0.5 * (B + B.transpose(0, 2, 1))
    C = spread(rng, nao, nocc, spread=6)
    return B, C


def _build_modes(df, B, C, s, modes=(0, 2)):
    Cg = cuda(C)
    out = {}
    for mode in modes:
        ctx, _ = _ctx(df, B, C.shape[1])
        ctx.set_cluster_pairs(mode)
        K = ctx.build_K(Cg, s)[0] if np.isscalar(s) else ctx.build_K_blocks(Cg, s)[0]
        out[mode] = K.cpu().numpy()
        ctx.sync_status()
    return out


@pytest.mark.parametrize("s", [3, 6])
def test_cluster_pairs_vs_oracle(df, s):
    # nocc 140: two occupied-orbital tiles (the second ragged) pair in the
    # first GEMM; nao 160: two AO tiles, so the second GEMM's pair at j = 0
    # also computes the lower tile; naux 24: one ragged auxiliary block
    B, C = _random_df(11, 24, 160, 140)
    out = _build_modes(df, B, C, s, modes=(0, 1, 2))
    assert np.array_equal(out[0], out[2]) and np.array_equal(out[1], out[2])
    ref = O.emulated_exchange(B, C, s)
    if s <= 5:
        assert np.array_equal(out[2], ref)
    else:
        assert np.max(np.abs(out[2] - ref)) <= 1e-14 * np.max(np.abs(ref))
    assert np.array_equal(out[2], out[2].T)


def test_cluster_pairs_odd_tile_count(df):
    # nao 300: three AO tiles, so the second tile of one pair lies past the
    # last one (it reads zeros and stores nothing)
    B, C = _random_df(12, 16, 300, 20)
    out = _build_modes(df, B, C, 5)
    assert np.array_equal(out[0], out[2])
    assert np.array_equal(out[2], O.emulated_exchange(B, C, 5))


def test_cluster_pairs_block_slices(df):
    # two auxiliary blocks (128 + 2 functions) with their own slice counts
    B, C = _random_df(13, 130, 140, 6)
    out = _build_modes(df, B, C, [5, 3])
    assert np.array_equal(out[0], out[2])
    assert np.array_equal(out[2], O.emulated_exchange(B, C, [5, 3]))


@pytest.mark.parametrize("w", [inputs.Workload("df-40atom-nao200-naux600-nocc150", 40, 150, 7000),
                               inputs.Workload("df-60atom-nao300-naux900-nocc120", 60, 120, 7100)])
def test_cluster_pairs_physical_inputs(df, w):
    mol, B, C, D = inputs.make_inputs(w)
    for s in (5, 8):
        out = _build_modes(df, B, C, s)
        assert np.array_equal(out[0], out[2])


def test_cluster_pairs_option_is_checked(df, small):
    B, C, D = small
    ctx, _ = _ctx(df, B, C.shape[1])
    for bad in (-1, 3):
        with pytest.raises(df.DFError):
            ctx.set_cluster_pairs(bad)


def test_exchange_zero_rows(df, small):
    # AO functions 0 and 7 removed from B: the rows (block, mu) of X for them
    # are zero in every block, so the first GEMM records no exponent bound for
    # them, the X split takes exponent 0 and zero digits, and K's rows and
    # columns 0 and 7 are zero
    B, C, D = small
    B = B.copy()
    for mu in (0, 7):
        B[:, mu, :] = 0.0
        B[:, :, mu] = 0.0
    ctx, _ = _ctx(df, B, C.shape[1])
    for s in (3, 5):
        K = ctx.build_K(cuda(C), s)[0].cpu().numpy()
        assert np.array_equal(K, O.emulated_exchange(B, C, s))
        assert not K[[0, 7]].any() and not K[:, [0, 7]].any()


@pytest.mark.parametrize("pairs", [1, 0])
@pytest.mark.parametrize("nocc", [15, 16])
def test_x_split_rows_above_their_bound(df, pairs, nocc):
    """Rows of X whose largest |X| reaches 127/128 2^E for the first GEMM's bound E: their
    exponent is E + 1, so the X split reads them a second time.  With C's columns the unit
    vectors e_i, X[P, mu, i] = B[P, mu, i] (digit-truncated); a planted |B| = 0.999 above
    |B| < 0.5 everywhere else puts every other mu row of each block at exponent 1 against a bound
    of 0.  Both first-GEMM layouts (bound per thread with pairs, per warp without), odd and even
    nocc; K bit-exact against the oracle's emulation."""
    rng = np.random.default_rng(300 + nocc)
    nao, naux = 64, 192
    B = rng.uniform(-0.5, 0.5, (naux, nao, nao))
    B = 0.5 * (B + B.transpose(0, 2, 1))
    for b0 in (0, 128):
        for mu in range(0, nao, 2):
            P, i = b0 + 5 + (mu % 7), mu % nocc
            v = 0.999 if (mu // 2) % 2 == 0 else -0.999
            B[P, mu, i] = B[P, i, mu] = v
    C = np.zeros((nao, nocc))
    C[np.arange(nocc), np.arange(nocc)] = 1.0
    ctx = df.Context(nao, naux, nocc)
    ctx.set_cluster_pairs(pairs)
    Bg = cuda(B)
    ctx.setup(Bg)
    for s in (3, 5):
        K = ctx.build_K(cuda(C), s)[0].cpu().numpy()
        assert np.array_equal(K, O.emulated_exchange(B, C, s))
    ctx.sync_status()


@pytest.mark.parametrize("nocc", [19, 20])
def test_exchange_odd_and_even_nocc(df, small, nocc):
    # the X split's scalar path (odd nocc) and its two-orbital path (even nocc)
    B, C, D = small
    C = np.ascontiguousarray(C[:, :nocc])
    ctx, _ = _ctx(df, B, nocc)
    for s in (4, 5):
        K = ctx.build_K(cuda(C), s)[0].cpu().numpy()
        assert np.array_equal(K, O.emulated_exchange(B, C, s))
    ctx.sync_status()


def test_setup_from_integrals(df, small):
    # B = L^{-1} (P|mu nu) on the device against the oracle's own Cholesky and
    # forward substitution, within the forward-error bound n u sqrt(cond V) |B|
    mol = inputs.molecule(inputs.SMALL.n_atoms, inputs.SMALL.seed)
    T = inputs.int3c(mol)
    V = inputs.metric(mol)
    Bo = O.df_tensor(T, V)
    ctx = df.Context(mol.nao, mol.naux, 20)
    Bg = ctx.setup_integrals(cuda(T), cuda(V)).cpu().numpy()
    tol = V.shape[0] * 2.0 ** -52 * math.sqrt(np.linalg.cond(V)) * np.max(np.abs(Bo))
    assert np.max(np.abs(Bg - Bo)) <= tol
    assert np.array_equal(Bg, Bg.transpose(0, 2, 1))
    # the attached B drives the builds: K is the oracle's emulation of that B
    B, C, D = small
    K = ctx.build_K(cuda(C), 5)[0].cpu().numpy()
    assert np.array_equal(K, O.emulated_exchange(Bg, C, 5))


def test_setup_from_integrals_rejects_indefinite_metric(df):
    naux, nao = 8, 4
    T = np.random.default_rng(3).standard_normal((naux, nao, nao))
    V = np.eye(naux)
    V[5, 5] = -1.0
    ctx = df.Context(nao, naux, 2)
    Tg = cuda(T)
    with pytest.raises(df.DFError) as e:
        ctx.setup_integrals(Tg, cuda(V))
    assert e.value.status == -4  # DF_ERR_NOT_PD
    assert np.array_equal(Tg.cpu().numpy(), T)


def test_bounded_wait_reports_a_timeout_and_the_context_survives(df, small):
    """Failure detection without a fault: a wait on a barrier nothing completes
    runs out after its limit, is reported as DF_ERR_TIMEOUT, and the next
    build on the same context is still correct."""
    import time
    t0 = time.perf_counter()
    assert df.selftest_wait_timeout(300) == -5
    dt = time.perf_counter() - t0
    assert 0.29 <= dt < 30.0
    B, C, D = small
    ctx, _ = _ctx(df, B, C.shape[1])
    K, _ = ctx.build_K(cuda(C), 0)
    ctx.sync_status()
    assert np.allclose(K.cpu().numpy(), O.exchange(B, C), rtol=0, atol=1e-12 * np.abs(O.exchange(B, C)).max())


def test_setup_rejects_an_asymmetric_tensor(df, small):
    """rho and J read the upper triangle of each B_P, so df_setup requires exact symmetry:
    one element off by one ulp is refused with DF_ERR_ARG; the symmetric tensor is taken."""
    B, C, D = small
    Bbad = B.copy()
    Bbad[7, 3, 11] = np.nextafter(Bbad[7, 3, 11], np.inf)
    ctx = df.Context(B.shape[1], B.shape[0], C.shape[1])
    with pytest.raises(df.DFError) as e:
        ctx.setup(cuda(Bbad))
    assert e.value.status == -1
    with pytest.raises(df.DFError):
        ctx.build_J(cuda(D))               # not set up: refused
    ctx.setup(cuda(B))
    J = ctx.build_J(cuda(D))[0].cpu().numpy()
    J_ref = O.coulomb(B, O.rho(B, D))
    assert np.max(np.abs(J - J_ref)) <= 1e-12 * np.max(np.abs(J_ref))
