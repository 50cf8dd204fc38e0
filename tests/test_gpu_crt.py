"""GPU parity of the CRT (Ozaki scheme II) emulated GEMM against its CPU oracle,
through the C ABI: residues, residue products and the reconstructed FP64
products are integer or correctly rounded results, so all are bit-exact."""
import numpy as np
import pytest
import torch

from oracle import crt_oracle as CO

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def df():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_08077_gb300 import build, df as dfmod
    build.build_all()
    return dfmod


def _mat(rng, rows, cols, spread=8.0, zero_row=None):
    A = rng.standard_normal((rows, cols)) * np.exp(rng.uniform(-spread, spread, (rows, 1)))
    A *= rng.random((rows, cols)) > 0.1                       # some exact zeros
    if zero_row is not None:
        A[zero_row] = 0.0
    return A


@pytest.mark.parametrize("rows,cols,nmod", [(37, 5, 2), (130, 333, 7), (64, 1200, 12), (9, 4097, 16)])
def test_residues_bitexact(df, rows, cols, nmod):
    rng = np.random.default_rng(rows + cols + nmod)
    A = _mat(rng, rows, cols, zero_row=3)
    q = CO.operand_bits(cols, nmod)
    assert q >= 2
    e_ref, Ai = CO.scaled_integers(A, q)
    e, R = df.crt_split_rows(torch.from_numpy(A).cuda(), nmod)
    assert np.array_equal(e.cpu().numpy(), e_ref)
    R = R.cpu().numpy()
    for i, m in enumerate(CO.moduli(nmod)):
        assert np.array_equal(R[i], CO.residues(Ai, m)), i


@pytest.mark.parametrize("M,N,K,nmod", [(300, 200, 333, 4), (129, 257, 64, 9), (260, 130, 2500, 16),
                                        (5, 3, 1, 3)])
def test_residue_products_bitexact(df, M, N, K, nmod):
    rng = np.random.default_rng(M * N + K)
    A = _mat(rng, M, K, zero_row=1)
    B = _mat(rng, N, K, spread=3.0)
    q = CO.operand_bits(K, nmod)
    ea_ref, Ai = CO.scaled_integers(A, q)
    eb_ref, Bi = CO.scaled_integers(B, q)
    Y_ref = CO.residue_products(Ai, Bi, CO.moduli(nmod))
    Y, ea, eb = df.crt_residue_products(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), nmod)
    assert np.array_equal(ea.cpu().numpy(), ea_ref) and np.array_equal(eb.cpu().numpy(), eb_ref)
    assert np.array_equal(Y.cpu().numpy(), Y_ref)


@pytest.mark.parametrize("M,N,K,nmod", [(260, 130, 200, 6), (133, 70, 1000, 12), (64, 40, 3000, 16),
                                        (200, 17, 77, 2)])
def test_emulated_gemm_crt_bitexact(df, M, N, K, nmod):
    rng = np.random.default_rng(7 * M + N + K)
    A = _mat(rng, M, K, zero_row=0)
    B = _mat(rng, N, K, spread=2.0, zero_row=2)
    ref = CO.emulated_gemm_crt(A, B, nmod)
    out = df.emulated_gemm_crt(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), nmod).cpu().numpy()
    assert np.array_equal(out, ref)


def test_integer_matrices_exact(df):
    rng = np.random.default_rng(5)
    A = rng.integers(-100, 101, (300, 130)).astype(np.float64) * 4.0
    B = rng.integers(-100, 101, (140, 130)).astype(np.float64) / 8.0
    out = df.emulated_gemm_crt(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 6).cpu().numpy()
    assert np.array_equal(out, A @ B.T)


@pytest.mark.parametrize("nmod", [8, 12, 15])
def test_large_within_bound_of_fp64(df, nmod):
    # a first-exchange-GEMM shape (rows (P, mu), K = nao, N = nocc): the error
    # against the FP64 product stays within the oracle's bound plus FP64 rounding
    torch.manual_seed(nmod)
    A = torch.randn(4096, 1200, dtype=torch.float64, device="cuda")
    A *= torch.exp(torch.empty(4096, 1, dtype=torch.float64, device="cuda").uniform_(-6, 6))
    B = torch.linalg.qr(torch.randn(1200, 250, dtype=torch.float64, device="cuda"))[0].T.contiguous()
    out = df.emulated_gemm_crt(A, B, nmod)
    ref = A @ B.T
    An, Bn = A.cpu().numpy(), B.cpu().numpy()
    o = out.cpu().numpy()
    bound = CO.error_bound(An, Bn, nmod) + 1200 * 2.0 ** -52 * (np.abs(An) @ np.abs(Bn).T) + np.spacing(np.abs(o))
    assert np.all(np.abs(o - ref.cpu().numpy()) <= bound)


def test_rejects_bad_arguments(df):
    A = torch.zeros(4, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(df.DFError) as e:
        df.emulated_gemm_crt(A, A, 17)
    assert e.value.status == -1
    with pytest.raises(df.DFError):
        df.emulated_gemm_crt(A, A, 1)


@pytest.mark.parametrize("nmod", [8, 13])
def test_gram_product_shares_one_split(df, nmod):
    # A B^T with B the same tensor as A (K_b = X_b X_b^T): one split on the device,
    # rows wider than 2048 (a whole block per row)
    rng = np.random.default_rng(40 + nmod)
    A = _mat(rng, 150, 2500, spread=5.0, zero_row=4)
    At = torch.from_numpy(A).cuda()
    out = df.emulated_gemm_crt(At, At, nmod).cpu().numpy()
    assert np.array_equal(out, CO.emulated_gemm_crt(A, A, nmod))
    assert np.array_equal(out, out.T)


@pytest.mark.parametrize("s", [3, 5])
def test_slice_gram_product_shares_one_split(df, s):
    from oracle import df_oracle as O
    rng = np.random.default_rng(60 + s)
    A = _mat(rng, 140, 2500, spread=5.0, zero_row=7)
    At = torch.from_numpy(A).cuda()
    out = df.emulated_gemm(At, At, s).cpu().numpy()
    assert np.array_equal(out, O.emulated_matmul(A, A.T, s))      # T = 0 here: bit-exact
    Bt = At.clone()                                                 # a different pointer: two splits
    assert np.array_equal(df.emulated_gemm(At, Bt, s).cpu().numpy(), out)
