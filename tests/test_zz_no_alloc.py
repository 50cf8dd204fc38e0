"""df_emulated_gemm_static: the emulated product without any device allocation.

Callers whose device memory is owned by a framework pool, or that cannot take
the synchronisation of cudaMalloc/cudaFree, use this entry point; its scratch
is a fixed static device array.  The tests call it through the C ABI twice in
a row (different shapes and slice counts, so the second call runs on the
scratch contents the first one left) and check each result against the CPU
oracle's emulated product (bit-exact where the fixed-point recombination is
exact, else within the bound of its dropped bits) and against the allocating
entry point df_emulated_gemm, which runs the same kernels: those two must be
identical.  A Gram product (the same matrix as both operands) takes the
one-split path of both entry points.  The device's free memory must not
change across a call once the array is mapped.  The documented size formula
is checked at the edge of the 32 MiB scratch: one shape just under it runs,
one just over it is refused with DF_ERR_SCRATCH and leaves the output as it
was.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import df_oracle as O

pytestmark = pytest.mark.gpu

DF_ERR_SCRATCH = -8
SCRATCH_BYTES = 32 << 20


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_08077_gb300 import build
    L = ctypes.CDLL(build.build_library())
    P, I = ctypes.c_void_p, ctypes.c_int
    for name in ("df_emulated_gemm", "df_emulated_gemm_static"):
        getattr(L, name).argtypes = [P, P, I, I, I, I, P, P]
    return L


def _call(L, name, A, B, s, out):
    M, K = A.shape
    N = B.shape[0]
    stream = torch.cuda.current_stream().cuda_stream
    return getattr(L, name)(A.data_ptr(), B.data_ptr(), M, N, K, s, out.data_ptr(), stream)


def _operand(rng, m, k):
    return rng.standard_normal((m, k)) * np.exp2(rng.integers(-12, 1, (m, k)))


def _shift_T(s, k):
    """Truncation of the int64 fixed-point sum (the library's rule)."""
    bound = sum((g + 1) * k * 16384 * 2 ** (8 * (s - 1 - g)) for g in range(s))
    bits = 0
    while 2 ** bits < bound:
        bits += 1
    return max(0, bits - 61)


def _check_vs_oracle(got, A, B, s):
    """Bit-exact against the oracle when the recombination keeps every bit (T = 0),
    else within the dropped bits' bound (half a unit per accumulation chunk)."""
    ref = O.emulated_matmul(A, B.T, s)
    K = A.shape[1]
    ktiles = -(-K // 64)
    T = _shift_T(s, ktiles * 64)
    if T == 0:
        assert np.array_equal(got, ref)
        return
    ea, eb = O.row_exponents(A), O.row_exponents(B)
    unit = np.ldexp(1.0, (ea[:, None] + eb[None, :] - 14 - 8 * (s - 1) + T).astype(np.int64))
    chunks = sum(-(-((g + 1) * ktiles) // 16) for g in range(s))
    assert np.all(np.abs(got - ref) <= unit * (0.5 * chunks + 1) + 2 * np.spacing(np.abs(ref)))


def test_static_scratch_matches_oracle_and_allocating_entry(lib):
    rng = np.random.default_rng(77)
    cases = [(300, 200, 700, 5), (130, 257, 1100, 8), (200, None, 700, 5)]   # None: B is A (Gram)
    for M, N, K, s in cases:
        A = _operand(rng, M, K)
        B = A if N is None else _operand(rng, N, K)
        Ag = torch.from_numpy(A).cuda()
        Bg = Ag if N is None else torch.from_numpy(B).cuda()
        n = B.shape[0]
        ref = torch.empty((M, n), dtype=torch.float64, device="cuda")
        got = torch.full((M, n), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, "df_emulated_gemm", Ag, Bg, s, ref) == 0
        assert _call(lib, "df_emulated_gemm_static", Ag, Bg, s, got) == 0
        assert torch.equal(got, ref)
        _check_vs_oracle(got.cpu().numpy(), A, B, s)


def test_static_scratch_allocates_nothing(lib):
    rng = np.random.default_rng(78)
    A = torch.from_numpy(_operand(rng, 260, 900)).cuda()
    B = torch.from_numpy(_operand(rng, 190, 900)).cuda()
    out = torch.empty((260, 190), dtype=torch.float64, device="cuda")
    assert _call(lib, "df_emulated_gemm_static", A, B, 6, out) == 0    # maps the array, loads the kernels
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for s in (6, 4):
        assert _call(lib, "df_emulated_gemm_static", A, B, s, out) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def _need(M, N, K, s):
    """The documented scratch size: 256-byte-rounded status word, exponents, digit planes."""
    r = lambda v: (v + 255) // 256 * 256  # noqa: E731
    ld = (K + 7) // 8 * 8
    return r(4) + r(4 * M) + r(4 * N) + r(2 * s * M * ld) + r(2 * s * N * ld)


def test_static_scratch_size_edge(lib):
    K, s = 1024, 8                      # 16 KiB of digits per row
    under, over = (1024, 1023), (1024, 1024)
    assert _need(*under, K, s) <= SCRATCH_BYTES < _need(*over, K, s)
    rng = np.random.default_rng(79)
    A = _operand(rng, 1024, K)
    Bh = _operand(rng, 1024, K)
    Ag = torch.from_numpy(A).cuda()
    Bg = torch.from_numpy(Bh).cuda()
    got = torch.empty((1024, 1023), dtype=torch.float64, device="cuda")
    ref = torch.empty_like(got)
    assert _call(lib, "df_emulated_gemm_static", Ag, Bg[:1023], s, got) == 0
    assert _call(lib, "df_emulated_gemm", Ag, Bg[:1023], s, ref) == 0
    assert torch.equal(got, ref)
    out = torch.full((1024, 1024), 3.0, dtype=torch.float64, device="cuda")
    assert _call(lib, "df_emulated_gemm_static", Ag, Bg, s, out) == DF_ERR_SCRATCH
    assert bool((out == 3.0).all())
    # a Gram product of the same 1024 rows needs one operand's planes only: it fits
    gram = torch.empty((1024, 1024), dtype=torch.float64, device="cuda")
    gram_ref = torch.empty_like(gram)
    assert _call(lib, "df_emulated_gemm_static", Ag, Ag, s, gram) == 0
    assert _call(lib, "df_emulated_gemm", Ag, Ag, s, gram_ref) == 0
    assert torch.equal(gram, gram_ref)


def test_static_scratch_refuses_oversize(lib):
    M = N = 2048
    K = 2048
    A = torch.zeros((M, K), dtype=torch.float64, device="cuda")
    B = torch.zeros((N, K), dtype=torch.float64, device="cuda")
    out = torch.full((M, N), 3.0, dtype=torch.float64, device="cuda")
    assert _call(lib, "df_emulated_gemm_static", A, B, 8, out) == DF_ERR_SCRATCH
    assert bool((out == 3.0).all())
