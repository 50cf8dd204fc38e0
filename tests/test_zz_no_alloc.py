"""df_emulated_gemm_static: the emulated product without any device allocation.

Callers whose device memory is owned by a framework pool, or that cannot take
the synchronisation of cudaMalloc/cudaFree, use this entry point; its scratch
is a fixed static device array.  The test calls it through the C ABI twice in
a row (different shapes and slice counts, so the second call runs on the
scratch contents the first one left) and checks each result against the
allocating entry point df_emulated_gemm, which runs the same kernels: the
results must be identical.  It also checks that a problem larger than the
scratch is refused with DF_ERR_SCRATCH and leaves the output untouched.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DF_ERR_SCRATCH = -8


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


def test_static_scratch_matches_allocating_entry(lib):
    rng = np.random.default_rng(77)
    cases = [(300, 200, 700, 5), (130, 257, 1100, 8)]
    for M, N, K, s in cases:
        A = torch.from_numpy(rng.standard_normal((M, K)) * np.exp2(rng.integers(-12, 1, (M, K)))).cuda()
        B = torch.from_numpy(rng.standard_normal((N, K)) * np.exp2(rng.integers(-12, 1, (N, K)))).cuda()
        ref = torch.empty((M, N), dtype=torch.float64, device="cuda")
        got = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, "df_emulated_gemm", A, B, s, ref) == 0
        assert _call(lib, "df_emulated_gemm_static", A, B, s, got) == 0
        assert torch.equal(got, ref)


def test_static_scratch_refuses_oversize(lib):
    M = N = 2048
    K = 2048
    A = torch.zeros((M, K), dtype=torch.float64, device="cuda")
    B = torch.zeros((N, K), dtype=torch.float64, device="cuda")
    out = torch.full((M, N), 3.0, dtype=torch.float64, device="cuda")
    assert _call(lib, "df_emulated_gemm_static", A, B, 8, out) == DF_ERR_SCRATCH
    assert bool((out == 3.0).all())
