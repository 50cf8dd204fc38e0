// The learned slice-count predictor: block features, a 16 -> 64 -> 64 -> 8
// MLP (FP32, ReLU, softmax over slice counts 1..8) with hand-written forward,
// backward and Adam kernels, and the label generator (per-block K error of
// the emulated build at every slice count against the native FP64 build).
//
// Parameter layout (one float buffer, row-major weights, y = W x + b):
//   W1 [64][16], b1 [64], W2 [64][64], b2 [64], W3 [8][64], b3 [8].
#include "df_ctx.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace {

constexpr int kIn = 16, kH = 64, kOut = 8;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kOut * kH, kNParams = oB3 + kOut;
static_assert(kNParams == 5768, "parameter count");

// One warp per row: forward pass; optionally keeps activations for backward.
__device__ __forceinline__ void mlp_row_forward(const float *__restrict__ P, const float *x, float *h1, float *h2,
                                                float *z, int lane) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = lane + 32 * r;
    float a = P[oB1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) a = fmaf(P[oW1 + j * kIn + k], x[k], a);
    h1[j] = a > 0.f ? a : 0.f;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = lane + 32 * r;
    float a = P[oB2 + j];
    for (int k = 0; k < kH; ++k) a = fmaf(P[oW2 + j * kH + k], h1[k], a);
    h2[j] = a > 0.f ? a : 0.f;
  }
  __syncwarp();
  if (lane < kOut) {
    float a = P[oB3 + lane];
    for (int k = 0; k < kH; ++k) a = fmaf(P[oW3 + lane * kH + k], h2[k], a);
    z[lane] = a;
  }
  __syncwarp();
}

__device__ __forceinline__ void softmax8(const float *z, float *p) {
  float m = z[0];
  for (int c = 1; c < kOut; ++c) m = fmaxf(m, z[c]);
  float s = 0.f;
  for (int c = 0; c < kOut; ++c) {
    p[c] = __expf(z[c] - m);
    s += p[c];
  }
  for (int c = 0; c < kOut; ++c) p[c] /= s;
}

constexpr int kRowsPerBlock = 8;

__global__ void __launch_bounds__(256) mlp_forward_kernel(const float *__restrict__ P, const float *__restrict__ X,
                                                          int n, float *__restrict__ probs) {
  __shared__ float sx[kRowsPerBlock][kIn], sh1[kRowsPerBlock][kH], sh2[kRowsPerBlock][kH], sz[kRowsPerBlock][kOut];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsPerBlock + w;
  if (row >= n) return;
  if (lane < kIn) sx[w][lane] = X[(long long)row * kIn + lane];
  __syncwarp();
  mlp_row_forward(P, sx[w], sh1[w], sh2[w], sz[w], lane);
  if (lane == 0) {
    float p[kOut];
    softmax8(sz[w], p);
    for (int c = 0; c < kOut; ++c) probs[(long long)row * kOut + c] = p[c];
  }
}

// Gradients of the mean cross-entropy (labels y in 0..7) summed into G, loss into *loss.
__global__ void __launch_bounds__(256) mlp_backward_kernel(const float *__restrict__ P, const float *__restrict__ X,
                                                           const int *__restrict__ y, int n, float *__restrict__ G,
                                                           float *__restrict__ loss) {
  __shared__ float sx[kRowsPerBlock][kIn], sh1[kRowsPerBlock][kH], sh2[kRowsPerBlock][kH], sz[kRowsPerBlock][kOut];
  __shared__ float sdz[kRowsPerBlock][kOut], sd2[kRowsPerBlock][kH], sd1[kRowsPerBlock][kH];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsPerBlock + w;
  if (row >= n) return;
  const float inv_n = 1.f / (float)n;
  if (lane < kIn) sx[w][lane] = X[(long long)row * kIn + lane];
  __syncwarp();
  mlp_row_forward(P, sx[w], sh1[w], sh2[w], sz[w], lane);
  if (lane == 0) {
    float p[kOut];
    softmax8(sz[w], p);
    const int yc = y[row];
    atomicAdd(loss, -logf(fmaxf(p[yc], 1e-30f)) * inv_n);
    for (int c = 0; c < kOut; ++c) sdz[w][c] = (p[c] - (c == yc ? 1.f : 0.f)) * inv_n;
  }
  __syncwarp();
  // layer 3
  if (lane < kOut) atomicAdd(&G[oB3 + lane], sdz[w][lane]);
  for (int idx = lane; idx < kOut * kH; idx += 32) {
    const int c = idx / kH, k = idx - c * kH;
    atomicAdd(&G[oW3 + idx], sdz[w][c] * sh2[w][k]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = lane + 32 * r;
    float a = 0.f;
    for (int c = 0; c < kOut; ++c) a = fmaf(P[oW3 + c * kH + j], sdz[w][c], a);
    sd2[w][j] = sh2[w][j] > 0.f ? a : 0.f;
  }
  __syncwarp();
  // layer 2
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = lane + 32 * r;
    atomicAdd(&G[oB2 + j], sd2[w][j]);
    for (int k = 0; k < kH; ++k) atomicAdd(&G[oW2 + j * kH + k], sd2[w][j] * sh1[w][k]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = lane + 32 * r;
    float a = 0.f;
    for (int c = 0; c < kH; ++c) a = fmaf(P[oW2 + c * kH + j], sd2[w][c], a);
    sd1[w][j] = sh1[w][j] > 0.f ? a : 0.f;
  }
  __syncwarp();
  // layer 1
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = lane + 32 * r;
    atomicAdd(&G[oB1 + j], sd1[w][j]);
    for (int k = 0; k < kIn; ++k) atomicAdd(&G[oW1 + j * kIn + k], sd1[w][j] * sx[w][k]);
  }
}

__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ m1,
                            float *__restrict__ m2, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float a = b1 * m1[i] + (1.f - b1) * g;
  const float v = b2 * m2[i] + (1.f - b2) * g * g;
  m1[i] = a;
  m2[i] = v;
  P[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

// ---- block features and labels ------------------------------------------------

// Static per-block statistics of B: [0] max|B|, [1] sum B^2, [2] sum of row
// exponents over nonzero rows, [3] nonzero rows, [4] min exponent, [5] max
// exponent, [6] rows with exponent < max_e - 20 (filled in a second pass).
// packed: B holds per P the upper triangle row by row (off-diagonal entries
// then count twice in the sum of squares).
__global__ void __launch_bounds__(256) block_stats_kernel(const double *__restrict__ B, const int *__restrict__ eB,
                                                          const int *__restrict__ perm, int naux, int nao,
                                                          double *__restrict__ stats, bool packed) {
  const int b = blockIdx.x;
  const int p0 = b * df::kBlock;
  const int nP = min(df::kBlock, naux - p0);
  const long long n2 = (long long)nao * nao;
  const long long npk = (long long)nao * (nao + 1) / 2;
  double mx = 0.0, ss = 0.0;
  for (int pl = 0; pl < nP; ++pl) {
    const int P = perm ? perm[p0 + pl] : p0 + pl;
    if (packed) {
      const double *src = B + (long long)P * npk;
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int mu = warp; mu < nao; mu += (int)(blockDim.x >> 5)) {
        const double *row = src + (long long)mu * nao - (long long)mu * (mu - 1) / 2 - mu;
        for (int nu = mu + lane; nu < nao; nu += 32) {
          const double v = row[nu];
          mx = fmax(mx, fabs(v));
          ss = fma(nu == mu ? v : 2.0 * v, v, ss);
        }
      }
    } else {
      const double *src = B + (long long)P * n2;
      for (long long i = threadIdx.x; i < n2; i += blockDim.x) {
        const double v = src[i];
        mx = fmax(mx, fabs(v));
        ss = fma(v, v, ss);
      }
    }
  }
  double esum = 0.0, cnt = 0.0, emin = 1e9, emax = -1e9;
  const int rows = nP * nao;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    const int e = eB[(long long)p0 * nao + r];
    // every row of the block counts (a zero row has exponent 0)
    esum += e;
    cnt += 1.0;
    emin = fmin(emin, (double)e);
    emax = fmax(emax, (double)e);
  }
  __shared__ double red[6][8];
  double vals[6] = {mx, ss, esum, cnt, emin, emax};
  for (int q = 0; q < 6; ++q) {
    double v = vals[q];
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = (q == 0 || q == 5) ? fmax(v, w) : (q == 4 ? fmin(v, w) : v + w);
    }
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 6; ++q) {
      double v = red[q][0];
      for (int k = 1; k < 8; ++k)
        v = (q == 0 || q == 5) ? fmax(v, red[q][k]) : (q == 4 ? fmin(v, red[q][k]) : v + red[q][k]);
      stats[b * 8 + q] = v;
    }
  }
  __syncthreads();
  // second pass: rows far below the block's largest row
  const int emx = (int)stats[b * 8 + 5];
  double small = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) small += (eB[(long long)p0 * nao + r] < emx - 20) ? 1.0 : 0.0;
  for (int o = 16; o > 0; o >>= 1) small += __shfl_xor_sync(0xffffffffu, small, o);
  __shared__ double rs[8];
  if ((threadIdx.x & 31) == 0) rs[threadIdx.x >> 5] = small;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < 8; ++k) v += rs[k];
    stats[b * 8 + 6] = v;
  }
}

// 16 features per block from the static statistics and the iteration's scalars.
// dD_dev, when given, replaces dD (the density change measured on the device).
__global__ void block_features_kernel(const double *__restrict__ stats, int nblk, int naux, int nao, int nocc,
                                      double tau, double dD, const double *__restrict__ dD_dev, double dE,
                                      int s_rule, float *__restrict__ F) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  if (dD_dev) dD = *dD_dev;
  if (!(dD >= 0.0 && dD <= 1e300)) dD = 1.0;  // a non-finite change reads as "large", never as NaN
  double gmax = 0.0, gss = 0.0;
  for (int k = 0; k < nblk; ++k) {
    gmax = fmax(gmax, stats[k * 8 + 0]);
    gss += stats[k * 8 + 1];
  }
  const double *st = stats + b * 8;
  const double tiny = 1e-300;
  const int nP = min(df::kBlock, naux - b * df::kBlock);
  float f[16];
  f[0] = (float)(log2(st[0] + tiny) / 32.0);
  f[1] = (float)(0.5 * log2(st[1] + tiny) / 32.0);
  f[2] = (float)(st[2] / fmax(st[3], 1.0) / 32.0);
  f[3] = (float)((st[5] - st[4]) / 32.0);
  f[4] = (float)(log10(tau) / 16.0);
  f[5] = (float)(log10(dD + 1e-30) / 16.0);
  f[6] = (float)((double)b / (double)nblk);
  f[7] = (float)(log2((double)nP) / 8.0);
  f[8] = (float)(log2((double)nao) / 12.0);
  f[9] = (float)(log2((double)nocc) / 10.0);
  f[10] = (float)(log2(st[1] / fmax(gss, tiny) + tiny) / 32.0);
  f[11] = (float)(st[6] / fmax(st[3], 1.0));
  f[12] = (float)(s_rule / 8.0);
  f[13] = (float)((log2(st[0] + tiny) - log2(gmax + tiny)) / 32.0);
  f[14] = (float)(log10(dE + 1e-30) / 16.0);
  f[15] = 1.0f;
  for (int k = 0; k < 16; ++k) F[b * 16 + k] = f[k];
}

// max over (mu <= nu) of |K_b(s) - K_b^FP64| per block b, from the second
// GEMM's int64 partials of the last emulated build (blocks of slice count s).
__global__ void block_error_kernel(const long long *__restrict__ Rp, const int *__restrict__ eX,
                                   const int *__restrict__ s_blk, df::ShiftTable T, const double *__restrict__ K64,
                                   int nao, int nblk, int nsplit, unsigned long long *__restrict__ err) {
  const int nu = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  const int b = blockIdx.z;
  if (nu >= nao || nu < mu) return;
  const long long bs = (long long)nao * nao;
  long long R = 0;
  for (int sp = 0; sp < nsplit; ++sp) R += Rp[((long long)b * nsplit + sp) * bs + (long long)nu * nao + mu];
  const int s = s_blk[b];
  const int k = eX[b * nao + mu] + eX[b * nao + nu] - 14 - 8 * (s - 1) + T.v[s];
  const double d = fabs(df::ldexp_i64(R, k) - K64[(long long)b * bs + (long long)mu * nao + nu]);
  atomicMax(&err[b], (unsigned long long)__double_as_longlong(d));
}

// Learned counts: per block the most probable class + 1, or s_rule when that
// probability is below min_conf (flag set); counts capped at s_max.
__global__ void pick_slices_kernel(const float *__restrict__ probs, int nblk, float min_conf, int s_rule, int s_max,
                                   int *__restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  int best = 0;
  float pb = probs[b * kOut];
  for (int c = 1; c < kOut; ++c)
    if (probs[b * kOut + c] > pb) {
      pb = probs[b * kOut + c];
      best = c;
    }
  const bool low = pb < min_conf;
  const int s = low ? s_rule : best + 1;
  out[b] = s < s_max ? s : s_max;
  out[nblk + b] = low ? 1 : 0;
}

// Exponents of the error-bound check: out[b] = max_mu eX[b, mu], out[nblk + b]
// = max eB over the block's (P, mu) rows, out[2 nblk] = max eC.  One CTA per
// block (plus one for eC).
__global__ void __launch_bounds__(256) check_exponents_kernel(const int *__restrict__ eX, const int *__restrict__ eB,
                                                              const int *__restrict__ eC, int nblk, int nao, int naux,
                                                              int nocc, int *__restrict__ out) {
  const int b = blockIdx.x;
  int ex = INT_MIN, eb = INT_MIN;
  if (b < nblk) {
    for (int mu = threadIdx.x; mu < nao; mu += blockDim.x) ex = max(ex, eX[b * nao + mu]);
    const long long r0 = (long long)b * df::kBlock * nao;
    const long long r1 = (long long)min(naux, (b + 1) * df::kBlock) * nao;
    for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) eb = max(eb, eB[r]);
  } else {
    for (int i = threadIdx.x; i < nocc; i += blockDim.x) ex = max(ex, eC[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
    eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, o));
  }
  __shared__ int rx[8], rb[8];
  if ((threadIdx.x & 31) == 0) {
    rx[threadIdx.x >> 5] = ex;
    rb[threadIdx.x >> 5] = eb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) {
      ex = max(ex, rx[w]);
      eb = max(eb, rb[w]);
    }
    if (b < nblk) {
      out[b] = ex;
      out[nblk + b] = eb;
    } else {
      out[2 * nblk] = ex;
    }
  }
}

}  // namespace

struct df_mlp {
  float *P = nullptr, *G = nullptr, *m1 = nullptr, *m2 = nullptr, *loss = nullptr;
  int t = 0;
};

extern "C" {

df_status df_mlp_create(df_mlp **out) {
  if (!out) return DF_ERR_ARG;
  df_mlp *m = new (std::nothrow) df_mlp();
  if (!m) return DF_ERR_OOM;
  cudaError_t e = cudaMalloc(&m->P, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->G, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->m1, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->m2, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->P, 0, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMemset(m->m1, 0, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMemset(m->m2, 0, sizeof(float) * kNParams);
  if (e != cudaSuccess) {
    df_mlp_destroy(m);
    return DF_ERR_CUDA;
  }
  *out = m;
  return DF_OK;
}

void df_mlp_destroy(df_mlp *m) {
  if (!m) return;
  cudaFree(m->P);
  cudaFree(m->G);
  cudaFree(m->m1);
  cudaFree(m->m2);
  cudaFree(m->loss);
  delete m;
}

int df_mlp_num_params(void) { return kNParams; }

df_status df_mlp_set_params(df_mlp *m, const float *host, int n) {
  if (!m || !host || n != kNParams) return DF_ERR_ARG;
  m->t = 0;
  cudaError_t e = cudaMemcpy(m->P, host, sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->m1, 0, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMemset(m->m2, 0, sizeof(float) * kNParams);
  return e == cudaSuccess ? DF_OK : DF_ERR_CUDA;
}

df_status df_mlp_get_params(const df_mlp *m, float *host, int n) {
  if (!m || !host || n != kNParams) return DF_ERR_ARG;
  return cudaMemcpy(host, m->P, sizeof(float) * n, cudaMemcpyDeviceToHost) == cudaSuccess ? DF_OK : DF_ERR_CUDA;
}

df_status df_mlp_forward(df_mlp *m, const float *X, int n, float *probs, void *stream) {
  if (!m || !X || !probs || n < 0) return DF_ERR_ARG;
  if (n == 0) return DF_OK;
  mlp_forward_kernel<<<(n + kRowsPerBlock - 1) / kRowsPerBlock, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      m->P, X, n, probs);
  return cudaGetLastError() == cudaSuccess ? DF_OK : DF_ERR_CUDA;
}

df_status df_mlp_gradients(df_mlp *m, const float *X, const int *y, int n, float *grad_host, float *loss_host,
                           void *stream) {
  if (!m || !X || !y || n <= 0) return DF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(m->G, 0, sizeof(float) * kNParams, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return DF_ERR_CUDA;
  mlp_backward_kernel<<<(n + kRowsPerBlock - 1) / kRowsPerBlock, 256, 0, st>>>(m->P, X, y, n, m->G, m->loss);
  if (cudaGetLastError() != cudaSuccess) return DF_ERR_CUDA;
  if (grad_host) e = cudaMemcpyAsync(grad_host, m->G, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && loss_host) e = cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && (grad_host || loss_host)) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? DF_OK : DF_ERR_CUDA;
}

df_status df_mlp_train_step(df_mlp *m, const float *X, const int *y, int n, float lr, float *loss_host,
                            void *stream) {
  df_status r = df_mlp_gradients(m, X, y, n, nullptr, nullptr, stream);
  if (r != DF_OK) return r;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)m->t), c2 = 1.f - powf(b2, (float)m->t);
  adam_kernel<<<(kNParams + 255) / 256, 256, 0, st>>>(m->P, m->G, m->m1, m->m2, kNParams, lr, b1, b2, 1e-8f, c1, c2);
  if (cudaGetLastError() != cudaSuccess) return DF_ERR_CUDA;
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return DF_ERR_CUDA;
  }
  return DF_OK;
}

df_status df_block_features(df_ctx *c, int nocc, double tau, double dD, double dE, int s_rule, float *F,
                            void *stream) {
  if (!c || !F || nocc <= 0 || !(tau > 0.0)) return DF_ERR_ARG;
  if (!c->ready) return DF_ERR_STATE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!c->bstats) {
    if (cudaMalloc(&c->bstats, sizeof(double) * 8 * c->nblk) != cudaSuccess) return DF_ERR_OOM;
    block_stats_kernel<<<c->nblk, 256, 0, st>>>(c->B, c->eB, c->perm, c->naux, c->nao, c->bstats, c->packed);
    if (cudaGetLastError() != cudaSuccess) return DF_ERR_CUDA;
  }
  block_features_kernel<<<(c->nblk + 127) / 128, 128, 0, st>>>(c->bstats, c->nblk, c->naux, c->nao, nocc, tau, dD,
                                                               nullptr, dE, s_rule, F);
  return cudaGetLastError() == cudaSuccess ? DF_OK : DF_ERR_CUDA;
}

df_status df_block_errors(df_ctx *c, const double *C, int nocc, double *err_host, double *kmax_host, void *stream) {
  if (!c || !C || !err_host || nocc <= 0 || nocc > c->nocc_max) return DF_ERR_ARG;
  if (!c->ready) return DF_ERR_STATE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nao = c->nao, nblk = c->nblk;
  const long long bs = (long long)nao * nao;
  double *K64 = nullptr, *Kfull = nullptr;
  unsigned long long *err = nullptr;
  df_status r = DF_OK;
  cudaError_t e = cudaMalloc(&K64, sizeof(double) * bs * nblk);
  if (e == cudaSuccess) e = cudaMalloc(&Kfull, sizeof(double) * bs);
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(unsigned long long) * nblk);
  if (e != cudaSuccess) r = DF_ERR_OOM;
  // FP64 reference: X^T by cuBLAS (as in the native build), then K_b = Xt_b^T Xt_b per block
  if (r == DF_OK) r = df_build_K(c, C, nocc, 0, Kfull, nullptr, stream);
  if (r == DF_OK) {
    // the FP64 build leaves X^T [mu][(P, i)] in the natural P order; a block of
    // the exchange order (df_setup_ordered) gathers its functions' columns first
    const double one = 1.0, zero = 0.0;
    const long long ldx = (long long)c->naux * nocc;
    const long long kbw = (long long)df::kBlock * nocc;
    double *Xg = nullptr;
    if (!c->perm_h.empty() && cudaMalloc(&Xg, sizeof(double) * nao * kbw) != cudaSuccess) r = DF_ERR_OOM;
    for (int b = 0; b < nblk && r == DF_OK; ++b) {
      const int nP = (b + 1) * df::kBlock <= c->naux ? df::kBlock : c->naux - b * df::kBlock;
      const double *Xb = c->X + (long long)b * df::kBlock * nocc;
      long long ld = ldx;
      if (Xg) {
        for (int j = 0; j < nP && r == DF_OK; ++j)
          if (cudaMemcpy2DAsync(Xg + (long long)j * nocc, sizeof(double) * kbw,
                                c->X + (long long)c->perm_h[b * df::kBlock + j] * nocc, sizeof(double) * ldx,
                                sizeof(double) * nocc, nao, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            r = DF_ERR_CUDA;
        Xb = Xg;
        ld = kbw;
      }
      if (r == DF_OK && cublasDgemm(c->cublas, CUBLAS_OP_T, CUBLAS_OP_N, nao, nao, nP * nocc, &one, Xb, (int)ld, Xb,
                                    (int)ld, &zero, K64 + (long long)b * bs, nao) != CUBLAS_STATUS_SUCCESS)
        r = DF_ERR_CUDA;
    }
    if (Xg) {
      cudaStreamSynchronize(st);
      cudaFree(Xg);
    }
  }
  if (r == DF_OK && kmax_host) {
    // max|K| of the FP64 build (host side, once)
    std::vector<double> h((size_t)bs);
    if (cudaMemcpyAsync(h.data(), Kfull, sizeof(double) * bs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      r = DF_ERR_CUDA;
    double mx = 0.0;
    for (double v : h) mx = fmax(mx, fabs(v));
    *kmax_host = mx;
  }
  std::vector<int> sb(nblk);
  std::vector<unsigned long long> eh(nblk);
  for (int s = 1; s <= c->s_max && r == DF_OK; ++s) {
    for (int b = 0; b < nblk; ++b) sb[b] = s;
    r = df_build_K_blocks(c, C, nocc, sb.data(), Kfull, nullptr, stream);
    if (r != DF_OK) break;
    df::ShiftTable tt;
    const long long kb = df::xdigit_ld(nocc);
    for (int q = 0; q <= 8; ++q) tt.v[q] = df::fixed_point_shift(q, kb);
    if (cudaMemsetAsync(err, 0, sizeof(unsigned long long) * nblk, st) != cudaSuccess) {
      r = DF_ERR_CUDA;
      break;
    }
    dim3 grid((nao + 127) / 128, nao, nblk);
    block_error_kernel<<<grid, 128, 0, st>>>(c->Rp, c->eX, c->sblk, tt, K64, nao, nblk, c->nsplit, err);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(eh.data(), err, sizeof(unsigned long long) * nblk, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      r = DF_ERR_CUDA;
      break;
    }
    for (int b = 0; b < nblk; ++b) {
      double d;
      std::memcpy(&d, &eh[b], sizeof(double));
      err_host[b * 8 + (s - 1)] = d;
    }
  }
  for (int s = c->s_max + 1; s <= 8 && r == DF_OK; ++s)
    for (int b = 0; b < nblk; ++b) err_host[b * 8 + (s - 1)] = err_host[b * 8 + (c->s_max - 1)];
  cudaStreamSynchronize(st);
  cudaFree(K64);
  cudaFree(Kfull);
  cudaFree(err);
  return r;
}

}  // extern "C"

namespace {

// Table 1's printed accuracy per level (levels 1..4), the tolerance feature.
constexpr double kLevelTau[5] = {0.0, 7.1e-15, 1.8e-12, 4.7e-10, 1.2e-7};

// log2 of the a-priori error bound beta_b(s) of block b's K_b (see
// df_set_predictor): kb 1.01 (s+1) 2^(-8s) (2^(2E) + 2 nao 2^(F+Ec+E)) + kb 2^(2E-52).
double log2_bound(int s, double kb, int nao, int E, int F, int Ec) {
  const double a = 2.0 * E, b = 1.0 + std::log2((double)nao) + F + Ec + E;
  const double hi = std::max(a, b);
  const double trunc = std::log2(1.01 * (s + 1)) - 8.0 * s + hi + std::log2(std::exp2(a - hi) + std::exp2(b - hi));
  const double round = a - 52.0;
  const double top = std::max(trunc, round);
  return std::log2(kb) + top + std::log2(std::exp2(trunc - top) + std::exp2(round - top));
}

df_status cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return DF_OK;
  return e == cudaErrorMemoryAllocation ? DF_ERR_OOM : DF_ERR_CUDA;
}

}  // namespace

namespace df {

df_status build_K_learned(df_ctx *c, const double *C, int nocc, double *K, df_kstats *stats, cudaStream_t st) {
  const int level = c->level;
  const int s_rule = level_count(c, level);
  if (level < 1 || level > 4 || s_rule < 1 || s_rule > c->s_max) return DF_ERR_ARG;
  const int nblk = c->nblk;
  cudaError_t e = cudaSuccess;
  if (!c->lF) e = cudaMalloc(&c->lF, sizeof(float) * 16 * nblk);
  if (e == cudaSuccess && !c->lprobs) e = cudaMalloc(&c->lprobs, sizeof(float) * kOut * nblk);
  if (e == cudaSuccess && !c->lpick) e = cudaMalloc(&c->lpick, sizeof(int) * 2 * nblk);
  if (e == cudaSuccess && !c->lexp) e = cudaMalloc(&c->lexp, sizeof(int) * (2 * nblk + 1));
  if (e == cudaSuccess && !c->lhost) e = cudaMallocHost(&c->lhost, sizeof(int) * (2 * nblk + 1));
  if (e == cudaSuccess && !c->bstats) {
    e = cudaMalloc(&c->bstats, sizeof(double) * 8 * nblk);
    if (e == cudaSuccess) {
      block_stats_kernel<<<nblk, 256, 0, st>>>(c->B, c->eB, c->perm, c->naux, c->nao, c->bstats, c->packed);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) return cuda_err(e);
  // 1. features -> network -> counts (with the low-confidence fallback)
  block_features_kernel<<<(nblk + 127) / 128, 128, 0, st>>>(c->bstats, nblk, c->naux, c->nao, nocc,
                                                            kLevelTau[level], 0.0, c->dD, c->dE_last, s_rule, c->lF);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    mlp_forward_kernel<<<(nblk + kRowsPerBlock - 1) / kRowsPerBlock, 256, 0, st>>>(c->pred->P, c->lF, nblk,
                                                                                     c->lprobs);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    pick_slices_kernel<<<(nblk + 127) / 128, 128, 0, st>>>(c->lprobs, nblk, c->min_conf, s_rule, c->s_max,
                                                           c->lpick);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->lhost, c->lpick, sizeof(int) * 2 * nblk, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(e);
  std::vector<int> sb(c->lhost, c->lhost + nblk);
  int low = 0;
  for (int b = 0; b < nblk; ++b) low += c->lhost[nblk + b];
  // a count above the level's only pays for another below it: with none below,
  // every block takes the level's count
  bool below = false;
  for (int b = 0; b < nblk; ++b) below = below || sb[b] < s_rule;
  if (!below)
    for (int b = 0; b < nblk; ++b) sb[b] = std::min(sb[b], s_rule);
  // 2. first GEMM and X split at the predicted counts (C split deep enough for s_rule)
  df_status r = k_front(c, C, nocc, sb.data(), s_rule, st);
  if (r != DF_OK) return r;
  // 3. the error-bound check from the exponents
  check_exponents_kernel<<<nblk + 1, 256, 0, st>>>(c->eX, c->eB, c->eC, nblk, c->nao, c->naux, nocc, c->lexp);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->lhost, c->lexp, sizeof(int) * (2 * nblk + 1), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(e);
  const int Ec = c->lhost[2 * nblk];
  std::vector<double> lb_rule(nblk), lb(nblk);
  double ref = -INFINITY;
  for (int b = 0; b < nblk; ++b) {
    const int nP = std::min(kBlock, c->naux - b * kBlock);
    const double kb = (double)nP * nocc;
    lb_rule[b] = log2_bound(s_rule, kb, c->nao, c->lhost[b], c->lhost[nblk + b], Ec);
    lb[b] = log2_bound(sb[b], kb, c->nao, c->lhost[b], c->lhost[nblk + b], Ec);
    ref = std::max(ref, lb_rule[b]);
  }
  // sums of 2^(log2 bound - ref), all <= nblk
  auto total = [&](const std::vector<double> &v) {
    double t = 0.0;
    for (double x : v) t += std::exp2(x - ref);
    return t;
  };
  const double budget = total(lb_rule);
  double have = total(lb);
  int raised = 0;
  while (have > budget * (1.0 + 1e-12)) {
    int pick = -1;
    for (int b = 0; b < nblk; ++b)
      if (sb[b] < s_rule && (pick < 0 || lb[b] > lb[pick])) pick = b;
    if (pick < 0) break;  // cannot happen: every block at >= s_rule meets the budget
    sb[pick] = s_rule;
    lb[pick] = lb_rule[pick];
    ++raised;
    have = total(lb);
  }
  if (raised) {
    // 4. recompute the first GEMM and the X split with the raised counts
    r = k_front(c, C, nocc, sb.data(), s_rule, st);
    if (r != DF_OK) return r;
  }
  r = k_back(c, nocc, K, st);
  if (r != DF_OK) return r;
  if (stats) {
    stats->nblk = nblk;
    long long pairs = 0;
    for (int b = 0; b < nblk; ++b) {
      if (b < 256) stats->slices[b] = sb[b];
      pairs += (long long)sb[b] * (sb[b] + 1) / 2;
    }
    stats->recomputed = raised;
    stats->fallback = 0;
    stats->low_confidence = low;
    stats->level = level;
    stats->slice_pairs = pairs;
    stats->bound_ratio = have / budget;
  }
  return DF_OK;
}

}  // namespace df

extern "C" df_status df_set_predictor(df_ctx *c, df_mlp *net, float min_conf) {
  if (!c || !(min_conf > 0.f && min_conf <= 1.f)) return DF_ERR_ARG;
  c->pred = net;
  c->min_conf = min_conf;
  return DF_OK;
}
