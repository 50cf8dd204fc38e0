// The DF tensor on the device (Eq. cderi): B = L^{-1} (P|mu nu) with
// L L^T = (P|Q), the metric's Cholesky factor.
//
// The factorisation is cuSOLVER's potrf and the triangular solve cuBLAS's
// trsm (library steps, FP64, run once per molecule); the exact per-P
// symmetrisation and everything after it (the digit split of df_setup) are
// this library's kernels.  Row-major (P|mu nu) [naux][nao*nao] is the
// column-major matrix T_cm [nao*nao x naux]; B = L^{-1} T becomes
// B_cm = T_cm L^{-T}, i.e. X L^T = T_cm solved from the right, in place.
#include "df_ctx.h"

#include <cusolverDn.h>

namespace {

df_status record_status(df_ctx *c, df_status s) {
  if (c && s != DF_OK && c->last == DF_OK) c->last = s;
  return s;
}

// B_P := (B_P + B_P^T) / 2 for every P, element pairs (mu < nu) written to
// both halves: the same two roundings as the host generator's, so a B that
// is symmetric up to the solver's rounding becomes exactly symmetric.
__global__ void symmetrize_kernel(double *__restrict__ B, int nao) {
  double *b = B + (long long)blockIdx.y * nao * nao;
  const long long n2 = (long long)nao * nao;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n2;
       idx += (long long)gridDim.x * blockDim.x) {
    const int mu = (int)(idx / nao), nu = (int)(idx - (long long)mu * nao);
    if (mu < nu) {
      const double v = 0.5 * (b[(long long)mu * nao + nu] + b[(long long)nu * nao + mu]);
      b[(long long)mu * nao + nu] = v;
      b[(long long)nu * nao + mu] = v;
    }
  }
}

}  // namespace

extern "C" df_status df_setup_integrals(df_ctx *c, double *T_dev, const double *V_dev, const int *perm_host,
                                        void *stream) {
  if (!c || !T_dev || !V_dev) return record_status(c, DF_ERR_ARG);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int naux = c->naux, nao = c->nao;
  if (!c->cusolver) {
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return record_status(c, DF_ERR_CUDA);
    c->cusolver = h;
  }
  if (!c->cublas && cublasCreate(&c->cublas) != CUBLAS_STATUS_SUCCESS) return record_status(c, DF_ERR_CUDA);
  cusolverDnHandle_t hs = reinterpret_cast<cusolverDnHandle_t>(c->cusolver);
  if (cusolverDnSetStream(hs, st) != CUSOLVER_STATUS_SUCCESS || cublasSetStream(c->cublas, st) != CUBLAS_STATUS_SUCCESS)
    return record_status(c, DF_ERR_CUDA);

  double *L = nullptr, *work = nullptr;
  int *info = nullptr;
  int lwork = 0, h_info = 0;
  df_status r = DF_OK;
  const size_t vbytes = sizeof(double) * (size_t)naux * naux;
  if (cudaMalloc(&L, vbytes) != cudaSuccess || cudaMalloc(&info, sizeof(int)) != cudaSuccess) r = DF_ERR_OOM;
  if (r == DF_OK && cudaMemcpyAsync(L, V_dev, vbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) r = DF_ERR_CUDA;
  if (r == DF_OK &&
      cusolverDnDpotrf_bufferSize(hs, CUBLAS_FILL_MODE_LOWER, naux, L, naux, &lwork) != CUSOLVER_STATUS_SUCCESS)
    r = DF_ERR_CUDA;
  if (r == DF_OK && cudaMalloc(&work, sizeof(double) * (size_t)(lwork > 0 ? lwork : 1)) != cudaSuccess) r = DF_ERR_OOM;
  if (r == DF_OK &&
      cusolverDnDpotrf(hs, CUBLAS_FILL_MODE_LOWER, naux, L, naux, work, lwork, info) != CUSOLVER_STATUS_SUCCESS)
    r = DF_ERR_CUDA;
  if (r == DF_OK && (cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess))
    r = DF_ERR_CUDA;
  if (r == DF_OK && h_info > 0) r = DF_ERR_NOT_PD;  // leading minor h_info is not positive
  if (r == DF_OK && h_info < 0) r = DF_ERR_ARG;
  if (r == DF_OK) {
    const double one = 1.0;
    if (cublasDtrsm_64(c->cublas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT,
                       (int64_t)nao * nao, (int64_t)naux, &one, L, (int64_t)naux, T_dev,
                       (int64_t)nao * nao) != CUBLAS_STATUS_SUCCESS)
      r = DF_ERR_CUDA;
  }
  if (r == DF_OK) {
    dim3 grid(16, (unsigned)naux);
    symmetrize_kernel<<<grid, 256, 0, st>>>(T_dev, nao);
    if (cudaGetLastError() != cudaSuccess) r = DF_ERR_CUDA;
  }
  // the frees wait for the work queued on the stream that uses the buffers
  if (cudaStreamSynchronize(st) != cudaSuccess && r == DF_OK) r = DF_ERR_CUDA;
  cudaFree(L);
  cudaFree(work);
  cudaFree(info);
  if (r != DF_OK) return record_status(c, r);
  return df_setup_ordered(c, T_dev, perm_host, stream);
}
