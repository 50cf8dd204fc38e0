// C ABI of libdf (include/df.h): the context, its workspaces and the build
// sequences of the DF Coulomb and exchange matrices.
//
// Exchange build at s slices (Section 3.2; blocked as Eqs. df-k-blk-1/2):
//   1. split C per column into s digit planes          (split kernel, HBM)
//   2. X^T tiles = C^T B^T over the B digit planes     (slice GEMM, tensor cores)
//   3. split X per (block, mu) row over (P in block, i) (split kernel, HBM)
//   4. per block K_b = X_b X_b^T on upper tiles        (slice GEMM, tensor cores)
//   5. K = sum_b K_b in block order, mirrored          (reduce kernel)
// The FP64 comparison build (nslices = 0) runs the same contractions through
// cuBLAS DGEMM (strided batched over P) and DSYRK.
#include "df_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "df_ctx.h"

#include <cusolverDn.h>

namespace {

using df::kBlock;

df_status record(df_ctx *c, df_status s) {
  if (c && s != DF_OK && c->last == DF_OK) c->last = s;
  return s;
}

df_status cuda_status(df_ctx *c, cudaError_t e) {
  if (e == cudaSuccess) return DF_OK;
  if (e == cudaErrorMemoryAllocation) return record(c, DF_ERR_OOM);
  return record(c, DF_ERR_CUDA);
}

// Records a start/stop event pair around a phase when profiling is on.
struct PhaseTimer {
  df_ctx *c;
  int phase;
  cudaStream_t st;
  cudaEvent_t e1 = nullptr;
  PhaseTimer(df_ctx *c_, int ph, cudaStream_t s) : c(c_), phase(ph), st(s) {
    if (c && c->profiling) {
      cudaEvent_t e0 = take();
      e1 = take();
      cudaEventRecord(e0, st);
      c->ev[phase].push_back({e0, e1});
    }
  }
  ~PhaseTimer() {
    if (e1) cudaEventRecord(e1, st);
  }
  cudaEvent_t take() {
    if (!c->pool.empty()) {
      cudaEvent_t e = c->pool.back();
      c->pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};

#define DF_TRY(ctx, expr)                          \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return cuda_status(ctx, _e); \
  } while (0)

template <typename T>
cudaError_t alloc(df_ctx *c, T **p, size_t count) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 256;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
  if (e == cudaSuccess) c->bytes += (int64_t)bytes;
  return e;
}

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Upload per-block slice counts if they changed.
df_status upload_slices(df_ctx *c, const int *sb, cudaStream_t st) {
  bool same = true;
  for (int b = 0; b < c->nblk; ++b) same &= (c->sblk_host[b] == sb[b]);
  if (same) return DF_OK;
  DF_TRY(c, cudaStreamSynchronize(st));  // the pinned mirror may still feed an earlier copy
  for (int b = 0; b < c->nblk; ++b) c->sblk_host[b] = sb[b];
  DF_TRY(c, cudaMemcpyAsync(c->sblk, c->sblk_host, sizeof(int) * c->nblk, cudaMemcpyHostToDevice, st));
  return DF_OK;
}

__global__ void mirror_lower_to_upper(double *K, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j < n && j > i) K[(long long)i * n + j] = K[(long long)j * n + i];
}

df_status build_K_fp64(df_ctx *c, const double *C, int nocc, double *K, cudaStream_t st) {
  if (!c->cublas) {
    if (cublasCreate(&c->cublas) != CUBLAS_STATUS_SUCCESS) return record(c, DF_ERR_CUDA);
  }
  if (cublasSetStream(c->cublas, st) != CUBLAS_STATUS_SUCCESS) return record(c, DF_ERR_CUDA);
  const double one = 1.0, zero = 0.0;
  const long long ldx = (long long)c->naux * nocc;
  // Xt[mu][(P, i)] = X[P][mu][i]: per P, the column-major nocc x nao block
  // C^T B_P lands at Xt + P*nocc with leading dimension naux*nocc.
  {
    PhaseTimer t(c, DF_PHASE_GEMM1, st);
    const long long n2 = (long long)c->nao * c->nao;
    if (!c->packed) {
      cublasStatus_t s1 = cublasDgemmStridedBatched(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, nocc, c->nao, c->nao, &one,
                                                    C, nocc, 0, c->B, c->nao, n2, &zero, c->X, (int)ldx, nocc,
                                                    c->naux);
      if (s1 != CUBLAS_STATUS_SUCCESS) return record(c, DF_ERR_CUDA);
    } else {
      // packed B: dense copies of up to ~1 GB of B_P at a time
      const int chunk = (int)std::max<long long>(1, std::min<long long>(c->naux, (1ll << 27) / n2));
      double *dense = nullptr;
      DF_TRY(c, cudaMallocAsync(reinterpret_cast<void **>(&dense), sizeof(double) * n2 * chunk, st));
      df_status rs = DF_OK;
      for (int P0 = 0; P0 < c->naux && rs == DF_OK; P0 += chunk) {
        const int nP = std::min(chunk, c->naux - P0);
        if (df::launch_unpack(c->B, P0, nP, c->nao, dense, st) != cudaSuccess ||
            cublasDgemmStridedBatched(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, nocc, c->nao, c->nao, &one, C, nocc, 0,
                                      dense, c->nao, n2, &zero, c->X + (long long)P0 * nocc, (int)ldx, nocc,
                                      nP) != CUBLAS_STATUS_SUCCESS)
          rs = DF_ERR_CUDA;
      }
      cudaFreeAsync(dense, st);
      if (rs != DF_OK) return record(c, rs);
    }
  }
  PhaseTimer t2(c, DF_PHASE_GEMM2, st);
  cublasStatus_t s2 = cublasDsyrk(c->cublas, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T, c->nao, (int)ldx, &one, c->X,
                                  (int)ldx, &zero, K, c->nao);
  if (s2 != CUBLAS_STATUS_SUCCESS) return record(c, DF_ERR_CUDA);
  dim3 grid((c->nao + 127) / 128, c->nao);
  mirror_lower_to_upper<<<grid, 128, 0, st>>>(K, c->nao);
  DF_TRY(c, cudaGetLastError());
  return DF_OK;
}

}  // namespace

namespace df {

df_status ctx_upload_slices(df_ctx *c, const int *sb, cudaStream_t st) { return upload_slices(c, sb, st); }

// Parameters and operand maps of the first exchange GEMM: X^T = C^T B^T (the
// orbitals on the MMA's M side), or, when CTA pairs are on and the orbitals
// fit one 128-row tile, X = B C with the (P, mu) rows on the M side (pairs of
// those tiles share the stacked C slices; nao even keeps a pair inside one
// auxiliary block, so both CTAs run the same slice count).  X lands as
// [(P, mu)][i] either way.
bool gemm1_setup(df_ctx *c, int nocc, SgParams &p, CUtensorMap &ta, CUtensorMap &tb, int swap) {
  const int nao = c->nao, naux = c->naux;
  const long long c_plane = (long long)c->nocc_max * c->ld_nao;
  const bool swapped =
      nocc <= kTile && ((swap == 1 && c->pair_mode >= 1 && (nao & 1) == 0) || swap == 2);
  if (swapped) {
    if (!make_tmap_bf16(&ta, c->Bd, nao, (long long)naux * nao, c->s_max, c->ld_nao,
                        (long long)naux * nao * c->ld_nao))
      return false;
    if (!make_tmap_bf16(&tb, c->Cd, nao, nocc, c->s_max, c->ld_nao, c_plane)) return false;
    std::memset(&p, 0, sizeof(p));
    p.layout = kLayoutXs;
    p.mode = kModeXs;
    p.nt_m = (int)(((long long)naux * nao + kTile - 1) / kTile);
    p.nt_n = (nocc + kTile - 1) / kTile;
    p.nunits = p.nt_m * p.nt_n;
    p.m_valid = naux * nao;
    p.n_valid = nocc;
    p.ktiles = (nao + kKTile - 1) / kKTile;
    p.nao = nao;
    p.nocc = nocc;
    p.nblk = c->nblk;
    p.naux = naux;
    p.s_blk = c->sblk;
    for (int q = 0; q <= 8; ++q) p.shiftT[q] = fixed_point_shift(q, (long long)p.ktiles * kKTile);
    p.ea = c->eB;
    p.eb = c->eC;
    p.out = c->X;
    p.out_ld = nocc;
    p.status = c->status;
    p.pair = c->pair_mode;
    p.kmask = use_mask_tile(c);
    p.rowE = c->rowE;
    return true;
  }
  if (!make_tmap_bf16(&ta, c->Cd, nao, nocc, c->s_max, c->ld_nao, c_plane)) return false;
  if (!make_tmap_bf16(&tb, c->Bd, nao, (long long)naux * nao, c->s_max, c->ld_nao, (long long)naux * nao * c->ld_nao))
    return false;
  std::memset(&p, 0, sizeof(p));
  p.layout = kLayoutX;
  p.mode = kModeX;
  p.nt_m = (nocc + kTile - 1) / kTile;
  p.nt_n = (int)(((long long)naux * nao + kTile - 1) / kTile);
  p.nunits = p.nt_m * p.nt_n;
  p.m_valid = nocc;
  p.n_valid = naux * nao;
  p.ktiles = (nao + kKTile - 1) / kKTile;
  p.nao = nao;
  p.nocc = nocc;
  p.nblk = c->nblk;
  p.naux = naux;
  p.s_blk = c->sblk;
  for (int q = 0; q <= 8; ++q) p.shiftT[q] = fixed_point_shift(q, (long long)p.ktiles * kKTile);
  p.ea = c->eC;
  p.eb = c->eB;
  p.out = c->X;
  p.out_ld = nocc;
  p.status = c->status;
  p.pair = c->pair_mode;
  p.kmask = use_mask_tile(c);
  p.rowE = c->rowE;
  return true;
}

// Parameters and operand map of the second exchange GEMM (K_b = X_b X_b^T).
bool gemm2_setup(df_ctx *c, int nocc, int nsplit, SgParams &q2, CUtensorMap &tx) {
  const int nao = c->nao, naux = c->naux;
  const long long kb_ld = round_up((long long)kBlock * nocc, 64);
  if (!make_tmap_bf16(&tx, c->Xd, kb_ld, nao, (long long)c->s_max * c->nblk, kb_ld, (long long)nao * kb_ld))
    return false;
  std::memset(&q2, 0, sizeof(q2));
  q2.layout = kLayoutKPart;
  q2.mode = kModeKPart;
  q2.nt_m = q2.nt_n = (nao + kTile - 1) / kTile;
  q2.nsplit = nsplit;
  q2.nunits = q2.nt_m * (q2.nt_m + 1) / 2 * c->nblk * nsplit;
  q2.m_valid = q2.n_valid = nao;
  q2.nao = nao;
  q2.nocc = nocc;
  q2.nblk = c->nblk;
  q2.naux = naux;
  q2.s_blk = c->sblk;
  for (int q = 0; q <= 8; ++q) q2.shiftT[q] = fixed_point_shift(q, kb_ld);
  q2.ea = c->eX;
  q2.eb = c->eX;
  q2.raw = c->Rp;
  q2.out_ld = nao;
  q2.out_blk = (long long)nao * nao;
  q2.status = c->status;
  q2.pair = c->pair_mode;
  return true;
}

long long xdigit_ld(int nocc) { return round_up((long long)kBlock * nocc, 64); }

}  // namespace df

namespace df {

df_status k_front(df_ctx *c, const double *C, int nocc, const int *sb, int c_planes, cudaStream_t st,
                  cudaEvent_t after_gemm1) {
  int smax = 0;
  for (int b = 0; b < c->nblk; ++b) {
    if (sb[b] < 1 || sb[b] > c->s_max) return record(c, DF_ERR_ARG);
    smax = sb[b] > smax ? sb[b] : smax;
  }
  if (c_planes < smax) c_planes = smax;
  if (c_planes > c->s_max) c_planes = c->s_max;
  df_status s = upload_slices(c, sb, st);
  if (s != DF_OK) return s;
  const int nao = c->nao, naux = c->naux;
  // 1. C -> digit planes [t][i][nu]
  const long long c_plane = (long long)c->nocc_max * c->ld_nao;
  {
    PhaseTimer t(c, DF_PHASE_SPLIT_C, st);
    DF_TRY(c, df::launch_split_cols_bf16(C, nao, nocc, c_planes, c->eC, c->Cd, c->ld_nao, c_plane, st));
  }
  // 2. X^T = C^T B^T
  df::SgParams p;
  CUtensorMap ta, tb;
  if (!df::gemm1_setup(c, nocc, p, ta, tb)) return record(c, DF_ERR_CUDA);
  DF_TRY(c, cudaMemsetAsync(c->rowE, 0x80, sizeof(int) * (size_t)c->nblk * nao, st));
  {
    PhaseTimer t(c, DF_PHASE_GEMM1, st);
    DF_TRY(c, df::launch_slice_gemm(p, ta, tb, st));
  }
  if (after_gemm1) DF_TRY(c, cudaEventRecord(after_gemm1, st));
  // 3. X -> per-(block, mu) digit planes
  const long long kb_ld = df::xdigit_ld(nocc);
  {
    PhaseTimer t(c, DF_PHASE_SPLIT_X, st);
    df::ShiftTable t1;
    for (int q = 0; q <= 8; ++q) t1.v[q] = p.shiftT[q];
    DF_TRY(c, df::launch_split_xblocks(reinterpret_cast<const long long *>(c->X), naux, nao, nocc, smax, c->eB,
                                       c->eC, c->sblk, t1, c->rowE, c->eX, c->Xd, kb_ld, c->nblk, st));
  }
  return DF_OK;
}

df_status k_back(df_ctx *c, int nocc, double *K, cudaStream_t st) {
  // 4. per-block K_b on upper tiles (exact int64 partials per K split)
  df::SgParams q2;
  CUtensorMap tx;
  if (!df::gemm2_setup(c, nocc, c->nsplit, q2, tx)) return record(c, DF_ERR_CUDA);
  {
    PhaseTimer t(c, DF_PHASE_GEMM2, st);
    DF_TRY(c, df::launch_slice_gemm(q2, tx, tx, st));
  }
  // 5. K = sum_b K_b
  {
    PhaseTimer t(c, DF_PHASE_REDUCE, st);
    df::ShiftTable tt;
    for (int q = 0; q <= 8; ++q) tt.v[q] = q2.shiftT[q];
    DF_TRY(c, df::launch_kpart_reduce(c->Rp, c->eX, c->sblk, tt, c->nao, c->nblk, c->nsplit, K, st));
  }
  return DF_OK;
}

int level_count(const df_ctx *c, int level) {
  const bool fp64 = (level == 0 && c->level0_slices == 0) || (c->fp64_from >= 0 && level <= c->fp64_from);
  return fp64 ? 0 : (level == 0 ? c->level0_slices : df_level_slices(level));
}

}  // namespace df

namespace {

void fill_stats(df_kstats *stats, const df_ctx *c, const int *sb, int level) {
  if (!stats) return;
  stats->nblk = c->nblk;
  long long pairs = 0;
  for (int b = 0; b < c->nblk; ++b) {
    if (b < 256) stats->slices[b] = sb ? sb[b] : 0;
    if (sb) pairs += (long long)sb[b] * (sb[b] + 1) / 2;
  }
  stats->recomputed = 0;
  stats->fallback = sb ? 0 : 1;
  stats->low_confidence = 0;
  stats->level = level;
  stats->slice_pairs = pairs;
  stats->bound_ratio = sb ? 1.0 : 0.0;
}

df_status build_K_emulated(df_ctx *c, const double *C, int nocc, const int *sb, double *K, df_kstats *stats,
                           cudaStream_t st, int level = -1) {
  df_status s = df::k_front(c, C, nocc, sb, 0, st);
  if (s == DF_OK) s = df::k_back(c, nocc, K, st);
  if (s == DF_OK) fill_stats(stats, c, sb, level);
  return s;
}

}  // namespace

extern "C" {

const char *df_strerror(df_status s) {
  switch (s) {
    case DF_OK: return "ok";
    case DF_ERR_ARG: return "invalid argument";
    case DF_ERR_CUDA: return "CUDA or cuBLAS call failed";
    case DF_ERR_OOM: return "device allocation failed";
    case DF_ERR_NOT_PD: return "metric not positive definite";
    case DF_ERR_TIMEOUT: return "bounded device wait ran out";
    case DF_ERR_TOL: return "result missed its tolerance";
    case DF_ERR_STATE: return "call out of order";
    case DF_ERR_SCRATCH: return "problem exceeds the 32 MiB static scratch of df_emulated_gemm_static";
  }
  return "unknown status";
}

int df_level_for(double dE_rel) {
  if (dE_rel >= 2e-6) return 4;
  if (dE_rel >= 5e-9) return 3;
  if (dE_rel >= 2e-11) return 2;
  if (dE_rel >= 7e-14) return 1;
  return 0;
}

int df_level_slices(int level) {
  // s = ceil((m_emu + 1) / 8) with m_emu = 23, 31, 39, 47 for levels 4..1
  static const int m_emu[5] = {0, 47, 39, 31, 23};
  if (level <= 0 || level > 4) return 0;
  return (m_emu[level] + 1 + 7) / 8;
}

df_status df_create(df_ctx **out, int nao, int naux, int nocc_max, int s_max) {
  if (!out || nao <= 0 || naux <= 0 || nocc_max <= 0 || s_max < 1 || s_max > DF_S_MAX) return DF_ERR_ARG;
  *out = nullptr;
  df_ctx *c = new (std::nothrow) df_ctx();
  if (!c) return DF_ERR_OOM;
  c->nao = nao;
  c->naux = naux;
  c->nocc_max = nocc_max;
  c->s_max = s_max;
  c->nblk = (naux + kBlock - 1) / kBlock;
  c->ld_nao = round_up(nao, 8);
  c->kb_ld_max = round_up((long long)kBlock * nocc_max, 64);
  const long long rowsB = (long long)naux * nao;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = alloc(c, &c->Bd, (size_t)s_max * rowsB * c->ld_nao);
  if (e == cudaSuccess) e = alloc(c, &c->eB, (size_t)rowsB);
  if (e == cudaSuccess) e = alloc(c, &c->Cd, (size_t)s_max * nocc_max * c->ld_nao);
  if (e == cudaSuccess) e = alloc(c, &c->eC, (size_t)nocc_max);
  if (e == cudaSuccess) e = alloc(c, &c->X, (size_t)rowsB * nocc_max);
  if (e == cudaSuccess) e = alloc(c, &c->Xd, (size_t)s_max * c->nblk * nao * c->kb_ld_max);
  if (e == cudaSuccess) e = alloc(c, &c->eX, (size_t)c->nblk * nao);
  if (e == cudaSuccess) e = alloc(c, &c->rowE, (size_t)c->nblk * nao);
  {
    // split the K range of each block so that the second GEMM's units fill
    // whole waves of the persistent grid: the smallest split (fewest partials)
    // with at least one wave and a last wave >= 96 % full, else the fullest
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int nt = (nao + df::kTile - 1) / df::kTile;
    const long long units = (long long)nt * (nt + 1) / 2 * c->nblk;
    int best = 1;
    double best_eff = -1.0;
    for (int ns = 1; ns <= 8; ++ns) {
      const double waves = (double)(units * ns) / nsm;
      const double eff = waves < 1.0 ? waves : waves / std::ceil(waves);
      if (eff >= 0.96) {
        best = ns;
        break;
      }
      if (eff > best_eff + 1e-9) {
        best_eff = eff;
        best = ns;
      }
    }
    c->nsplit = best;
    c->nsm = nsm;
  }
  if (e == cudaSuccess) e = alloc(c, &c->Rp, (size_t)c->nblk * c->nsplit * nao * nao);
  if (e == cudaSuccess) e = alloc(c, &c->rho, (size_t)naux);
  if (e == cudaSuccess) e = alloc(c, &c->jk_work, (size_t)2);
  if (e == cudaSuccess) e = alloc(c, &c->epart, (size_t)3 * 296);
  if (e == cudaSuccess) e = alloc(c, &c->E, (size_t)4);
  if (e == cudaSuccess) e = alloc(c, &c->sblk, (size_t)c->nblk);
  if (e == cudaSuccess) e = alloc(c, &c->status, (size_t)1);
  if (e == cudaSuccess) e = alloc(c, &c->Dprev, (size_t)nao * nao);
  if (e == cudaSuccess) e = alloc(c, &c->dD, (size_t)1);
  if (e == cudaSuccess) e = alloc(c, &c->dD_part, (size_t)df::kDensityChangeBlocks);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&c->sblk_host), sizeof(int) * c->nblk);
  if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int));
  if (e == cudaSuccess) {
    const double one = 1.0;  // no previous density yet: the density-change feature reads 1
    e = cudaMemcpy(c->dD, &one, sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(c->sblk, 0, sizeof(int) * c->nblk);
  if (e == cudaSuccess) std::memset(c->sblk_host, 0, sizeof(int) * c->nblk);
  if (e != cudaSuccess) {
    df_status s = e == cudaErrorMemoryAllocation ? DF_ERR_OOM : DF_ERR_CUDA;
    cudaGetLastError();
    df_destroy(c);
    return s;
  }
  *out = c;
  return DF_OK;
}

void df_destroy(df_ctx *c) {
  if (!c) return;
  cudaFree(c->Bd);
  cudaFree(c->eB);
  cudaFree(c->Cd);
  cudaFree(c->eC);
  cudaFree(c->X);
  cudaFree(c->Xd);
  cudaFree(c->eX);
  cudaFree(c->rowE);
  cudaFree(c->Rp);
  cudaFree(c->rho);
  cudaFree(c->jk_work);
  if (c->jk_stream) cudaStreamDestroy(c->jk_stream);
  if (c->jk_fork) cudaEventDestroy(c->jk_fork);
  if (c->jk_join) cudaEventDestroy(c->jk_join);
  cudaFree(c->epart);
  cudaFree(c->E);
  cudaFree(c->sblk);
  cudaFree(c->status);
  cudaFree(c->Dprev);
  cudaFree(c->dD);
  cudaFree(c->dD_part);
  cudaFree(c->lF);
  cudaFree(c->lprobs);
  cudaFree(c->lpick);
  cudaFree(c->lexp);
  if (c->lhost) cudaFreeHost(c->lhost);
  cudaFree(c->bstats);
  cudaFree(c->mask_mu);
  cudaFree(c->mask_tile);
  cudaFree(c->perm);
  if (c->sblk_host) cudaFreeHost(c->sblk_host);
  for (int ph = 0; ph < DF_NPHASES; ++ph)
    for (auto &pr : c->ev[ph]) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->cublas) cublasDestroy(c->cublas);
  if (c->cusolver) cusolverDnDestroy(reinterpret_cast<cusolverDnHandle_t>(c->cusolver));
  delete c;
}

int64_t df_workspace_bytes(const df_ctx *c) { return c ? c->bytes : 0; }

df_status df_sparsity(const df_ctx *c, double *frac_ktiles, double *frac_chunks) {
  if (!c || !frac_ktiles || !frac_chunks) return DF_ERR_ARG;
  if (!c->ready) return DF_ERR_STATE;
  *frac_ktiles = c->frac_ktiles;
  *frac_chunks = c->frac_chunks;
  return DF_OK;
}

df_status df_set_profiling(df_ctx *c, int on) {
  if (!c) return DF_ERR_ARG;
  c->profiling = on != 0;
  return DF_OK;
}

df_status df_set_option(df_ctx *c, int option, int value) {
  if (!c) return DF_ERR_ARG;
  switch (option) {
    case DF_OPT_CLUSTER_PAIRS:
      if (value < 0 || value > 2) return DF_ERR_ARG;
      c->pair_mode = value;
      return DF_OK;
    case DF_OPT_SPARSE:
      if (value < 0 || value > 1) return DF_ERR_ARG;
      c->sparse_opt = value;
      return DF_OK;
    case DF_OPT_JK_OVERLAP:
      if (value < 0 || value > 4) return DF_ERR_ARG;
      c->jk_ctas = value;
      return DF_OK;
  }
  return DF_ERR_ARG;
}

df_status df_phase_times(df_ctx *c, double *ms, int *count) {
  if (!c || !ms || !count) return DF_ERR_ARG;
  df_status rs = DF_OK;
  for (int ph = 0; ph < DF_NPHASES; ++ph) {
    double total = 0.0;
    for (auto &pr : c->ev[ph]) {
      float t = 0.f;
      if (cudaEventSynchronize(pr.second) != cudaSuccess || cudaEventElapsedTime(&t, pr.first, pr.second) != cudaSuccess)
        rs = record(c, DF_ERR_CUDA);
      total += t;
      c->pool.push_back(pr.first);
      c->pool.push_back(pr.second);
    }
    ms[ph] = total;
    count[ph] = (int)c->ev[ph].size();
    c->ev[ph].clear();
  }
  return rs;
}

df_status df_last_error(const df_ctx *c) { return c ? c->last : DF_ERR_ARG; }

df_status df_setup(df_ctx *c, const double *B_dev, void *stream) { return df_setup_ordered(c, B_dev, nullptr, stream); }

namespace {

// df_setup_ordered / df_setup_packed: attach B (dense, or packed upper
// triangles), check it, split it and find its block sparsity.
df_status setup_common(df_ctx *c, const double *B_dev, const int *perm_host, bool packed, void *stream) {
  if (!c || !B_dev) return record(c, DF_ERR_ARG);
  cudaStream_t st = as_stream(stream);
  c->B = B_dev;
  c->packed = packed;
  if (perm_host) {
    std::vector<char> seen(c->naux, 0);
    for (int i = 0; i < c->naux; ++i) {
      if (perm_host[i] < 0 || perm_host[i] >= c->naux || seen[perm_host[i]]) return record(c, DF_ERR_ARG);
      seen[perm_host[i]] = 1;
    }
    if (!c->perm) DF_TRY(c, cudaMalloc(&c->perm, sizeof(int) * c->naux));
    DF_TRY(c, cudaMemcpy(c->perm, perm_host, sizeof(int) * c->naux, cudaMemcpyHostToDevice));
    c->perm_h.assign(perm_host, perm_host + c->naux);
  } else if (c->perm) {
    cudaFree(c->perm);
    c->perm = nullptr;
    c->perm_h.clear();
  }
  if (c->bstats) {
    cudaFree(c->bstats);
    c->bstats = nullptr;
  }
  c->ready = false;
  // rho and J read the upper triangle of each B_P: a dense B_P must be exactly symmetric
  if (!packed) {
    int h = 0;
    DF_TRY(c, df::launch_symmetry_check(B_dev, c->naux, c->nao, c->status, st));
    DF_TRY(c, cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DF_TRY(c, cudaStreamSynchronize(st));
    DF_TRY(c, cudaMemsetAsync(c->status, 0, sizeof(int), st));
    if (h) return record(c, DF_ERR_ARG);
  }
  const long long rows = (long long)c->naux * c->nao;
  if (packed)
    DF_TRY(c, df::launch_split_rows_packed(B_dev, c->naux, c->nao, c->s_max, c->eB, c->Bd, c->ld_nao,
                                           rows * c->ld_nao, c->perm, st));
  else
    DF_TRY(c, df::launch_split_rows_bf16(B_dev, rows, c->nao, c->nao, c->s_max, c->eB, c->Bd, c->ld_nao,
                                         rows * c->ld_nao, st, c->perm, c->nao));
  // block sparsity of a screened B (Section 2.1): exact zero chunks of the AO pairs
  c->sparse = false;
  c->frac_ktiles = c->frac_chunks = 1.0;
  if (c->nao <= 32 * df::kKTile) {
    const int ntiles = (int)((rows + df::kTile - 1) / df::kTile);
    if (!c->mask_mu) DF_TRY(c, cudaMalloc(&c->mask_mu, sizeof(uint32_t) * c->nao));
    if (!c->mask_tile) DF_TRY(c, cudaMalloc(&c->mask_tile, sizeof(uint32_t) * ntiles));
    if (packed)
      DF_TRY(c, df::launch_pair_masks_packed(B_dev, c->naux, c->nao, c->mask_mu, c->mask_tile, st));
    else
      DF_TRY(c, df::launch_pair_masks(B_dev, c->naux, c->nao, c->mask_mu, c->mask_tile, st));
    std::vector<uint32_t> mu(c->nao), tiles(ntiles);
    DF_TRY(c, cudaMemcpyAsync(mu.data(), c->mask_mu, sizeof(uint32_t) * c->nao, cudaMemcpyDeviceToHost, st));
    DF_TRY(c, cudaMemcpyAsync(tiles.data(), c->mask_tile, sizeof(uint32_t) * ntiles, cudaMemcpyDeviceToHost, st));
    DF_TRY(c, cudaStreamSynchronize(st));
    const int nk = (c->nao + df::kKTile - 1) / df::kKTile;
    long long on = 0, all = 0, kon = 0;
    for (int m = 0; m < c->nao; ++m)
      for (int k = m / df::kKTile; k < nk; ++k) {
        ++all;
        on += (mu[m] >> k) & 1u;
      }
    for (uint32_t t : tiles) kon += __builtin_popcount(t);
    c->frac_chunks = all ? (double)on / all : 1.0;
    c->frac_ktiles = (double)kon / ((double)ntiles * nk);
    c->sparse = on < all;
  }
  c->ready = true;
  return DF_OK;
}

}  // namespace

df_status df_setup_ordered(df_ctx *c, const double *B_dev, const int *perm_host, void *stream) {
  return setup_common(c, B_dev, perm_host, false, stream);
}

df_status df_setup_packed(df_ctx *c, const double *Bp_dev, const int *perm_host, void *stream) {
  return setup_common(c, Bp_dev, perm_host, true, stream);
}

df_status df_build_J(df_ctx *c, const double *D, double *J, double *rho, void *stream) {
  if (!c || !D || !J) return record(c, DF_ERR_ARG);
  if (!c->ready) return record(c, DF_ERR_STATE);
  cudaStream_t st = as_stream(stream);
  double *r = rho ? rho : c->rho;
  {
    PhaseTimer t(c, DF_PHASE_RHO, st);
    DF_TRY(c, df::launch_rho(c->B, D, c->naux, c->nao, r, st, df::use_mask_mu(c), c->packed, nullptr, 0, c->sparse));
  }
  {
    PhaseTimer t(c, DF_PHASE_COULOMB, st);
    DF_TRY(c, df::launch_coulomb(c->B, r, c->naux, c->nao, J, st, df::use_mask_mu(c), c->packed));
  }
  if (rho && rho != c->rho)
    DF_TRY(c, cudaMemcpyAsync(c->rho, rho, sizeof(double) * c->naux, cudaMemcpyDeviceToDevice, st));
  // the density change since the last Coulomb build (an input of the learned slice counts)
  DF_TRY(c, df::launch_density_change(D, c->Dprev, c->have_Dprev, (long long)c->nao * c->nao, c->dD_part, c->dD, st));
  c->have_Dprev = true;
  return DF_OK;
}

namespace {

// The internal stream and events of df_build_JK (created on first use).
df_status jk_streams(df_ctx *c) {
  if (c->jk_stream) return DF_OK;
  int lo = 0, hi = 0;
  DF_TRY(c, cudaDeviceGetStreamPriorityRange(&lo, &hi));
  DF_TRY(c, cudaStreamCreateWithPriority(&c->jk_stream, cudaStreamNonBlocking, hi));
  DF_TRY(c, cudaEventCreateWithFlags(&c->jk_fork, cudaEventDisableTiming));
  DF_TRY(c, cudaEventCreateWithFlags(&c->jk_join, cudaEventDisableTiming));
  return DF_OK;
}

}  // namespace

df_status df_build_JK(df_ctx *c, const double *D, const double *C, int nocc, int nslices, double *J, double *rho,
                      double *K, df_kstats *stats, void *stream) {
  if (!c || !D || !J || !C || !K || nocc <= 0 || nocc > c->nocc_max || nslices < -2 || nslices > c->s_max)
    return record(c, DF_ERR_ARG);
  if (!c->ready) return record(c, DF_ERR_STATE);
  int level = -1, s = nslices;
  if (s < 0) {
    level = c->level;
    s = df::level_count(c, level);
  }
  if (s > c->s_max) return record(c, DF_ERR_ARG);
  // the native FP64 build, the learned counts, a block-sparse B (whose
  // masked kernels take more registers than an SM shared with the X split
  // leaves) and the no-overlap option run the two builds one after the other
  if (c->jk_ctas == 0 || s == 0 || (nslices == -2 && c->level > 0) || df::use_mask_mu(c)) {
    df_status r = df_build_J(c, D, J, rho, stream);
    return r == DF_OK ? df_build_K(c, C, nocc, nslices, K, stats, stream) : r;
  }
  df_status r = jk_streams(c);
  if (r != DF_OK) return r;
  cudaStream_t st = as_stream(stream), side = c->jk_stream;
  int sb[4096];
  if (c->nblk > 4096) return record(c, DF_ERR_ARG);
  for (int b = 0; b < c->nblk; ++b) sb[b] = s;
  // the exchange front (C split, first GEMM, X split) in the caller's stream;
  // the Coulomb build forks after the first GEMM, whose persistent grid fills
  // every SM, and runs beside the X split: rho and J are bound by the FP64
  // pipe, the X split by HBM and integer work, so they share the SMs
  r = df::k_front(c, C, nocc, sb, 0, st, c->jk_fork);
  if (r != DF_OK) return r;
  DF_TRY(c, cudaStreamWaitEvent(side, c->jk_fork, 0));
  double *rr = rho ? rho : c->rho;
  const int grid = c->jk_ctas * (c->nsm > 0 ? c->nsm : 1);
  DF_TRY(c, cudaMemsetAsync(c->jk_work, 0, 2 * sizeof(int), side));
  {
    PhaseTimer t(c, DF_PHASE_RHO, side);
    DF_TRY(c, df::launch_rho(c->B, D, c->naux, c->nao, rr, side, nullptr, c->packed, c->jk_work, grid, c->sparse));
  }
  {
    PhaseTimer t(c, DF_PHASE_COULOMB, side);
    DF_TRY(c, df::launch_coulomb(c->B, rr, c->naux, c->nao, J, side, nullptr, c->packed, c->jk_work + 1, grid));
  }
  if (rho && rho != c->rho)
    DF_TRY(c, cudaMemcpyAsync(c->rho, rho, sizeof(double) * c->naux, cudaMemcpyDeviceToDevice, side));
  DF_TRY(c, cudaEventRecord(c->jk_join, side));
  // the second GEMM's persistent grid waits for whole SMs: join first
  DF_TRY(c, cudaStreamWaitEvent(st, c->jk_join, 0));
  r = df::k_back(c, nocc, K, st);
  if (r != DF_OK) return r;
  DF_TRY(c, df::launch_density_change(D, c->Dprev, c->have_Dprev, (long long)c->nao * c->nao, c->dD_part, c->dD, st));
  c->have_Dprev = true;
  fill_stats(stats, c, sb, level);
  return DF_OK;
}

df_status df_build_K(df_ctx *c, const double *C, int nocc, int nslices, double *K, df_kstats *stats, void *stream) {
  if (!c || !C || !K || nocc <= 0 || nocc > c->nocc_max || nslices < -2 || nslices > c->s_max)
    return record(c, DF_ERR_ARG);
  if (!c->ready) return record(c, DF_ERR_STATE);
  cudaStream_t st = as_stream(stream);
  int level = -1;
  if (nslices == -2 && c->level > 0) {
    if (!c->pred) return record(c, DF_ERR_STATE);
    return df::build_K_learned(c, C, nocc, K, stats, st);
  }
  if (nslices < 0) {
    // the adaptive rule's count for the current level (learned mode at level 0 likewise)
    level = c->level;
    nslices = df::level_count(c, level);
    if (nslices > c->s_max) return record(c, DF_ERR_ARG);
  }
  if (nslices == 0) {
    df_status s = build_K_fp64(c, C, nocc, K, st);
    if (s == DF_OK) fill_stats(stats, c, nullptr, level);
    return s;
  }
  int sb[4096];
  if (c->nblk > 4096) return record(c, DF_ERR_ARG);
  for (int b = 0; b < c->nblk; ++b) sb[b] = nslices;
  return build_K_emulated(c, C, nocc, sb, K, stats, st, level);
}

df_status df_build_K_blocks(df_ctx *c, const double *C, int nocc, const int *slices, double *K, df_kstats *stats,
                            void *stream) {
  if (!c || !C || !K || !slices || nocc <= 0 || nocc > c->nocc_max) return record(c, DF_ERR_ARG);
  if (!c->ready) return record(c, DF_ERR_STATE);
  return build_K_emulated(c, C, nocc, slices, K, stats, as_stream(stream));
}

df_status df_energy(df_ctx *c, const double *D, const double *J, const double *K, const double *rho, double *E_host,
                    void *stream) {
  if (!c || !D || !E_host) return record(c, DF_ERR_ARG);
  cudaStream_t st = as_stream(stream);
  const double *r = rho ? rho : c->rho;
  {
    PhaseTimer t(c, DF_PHASE_ENERGY, st);
    DF_TRY(c, df::launch_energy(D, J, K, r, c->nao, c->naux, c->epart, c->E, st));
  }
  DF_TRY(c, cudaMemcpyAsync(E_host, c->E, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  DF_TRY(c, cudaStreamSynchronize(st));
  return DF_OK;
}

df_status df_adaptive_reset(df_ctx *c, int fp64_from_level) {
  if (!c) return DF_ERR_ARG;
  c->level = 4;
  c->iter = 0;
  c->E_prev = 0.0;
  c->dE_last = 1.0;
  c->fp64_from = fp64_from_level;
  return DF_OK;
}

df_status df_adaptive_level0(df_ctx *c, int nslices) {
  if (!c || nslices < 0 || nslices > c->s_max) return DF_ERR_ARG;
  c->level0_slices = nslices;
  return DF_OK;
}

df_status df_adaptive_next(df_ctx *c, double energy, int *level_out, int *nslices_out) {
  if (!c || !level_out || !nslices_out) return DF_ERR_ARG;
  if (c->iter > 0 && energy != 0.0) {
    const double dE = std::fabs((energy - c->E_prev) / energy);
    c->dE_last = dE;
    const int lv = df_level_for(dE);
    if (lv < c->level) c->level = lv;  // precision never drops
  }
  c->E_prev = energy;
  c->iter += 1;
  *level_out = c->level;
  *nslices_out = df::level_count(c, c->level);
  return DF_OK;
}

df_status df_selftest_wait_timeout(int limit_ms, void *stream) {
  if (limit_ms < 1 || limit_ms > 10000) return DF_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  int *status = nullptr;
  int h = 0;
  cudaError_t e = cudaMalloc(&status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = df::launch_wait_selftest(status, (unsigned long long)limit_ms * 1000000ull, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (status) cudaFree(status);
  if (e != cudaSuccess) return DF_ERR_CUDA;
  return h == 1 ? DF_ERR_TIMEOUT : DF_OK;
}

df_status df_sync_status(df_ctx *c, void *stream) {
  if (!c) return DF_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  int h = 0;
  DF_TRY(c, cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  DF_TRY(c, cudaStreamSynchronize(st));
  if (h) {
    DF_TRY(c, cudaMemsetAsync(c->status, 0, sizeof(int), st));
    return record(c, DF_ERR_TIMEOUT);
  }
  return DF_OK;
}

df_status df_split_int8(const double *A, int rows, int cols, int ld, int nslices, int32_t *exps, int8_t *digits,
                        void *stream) {
  if (!A || !exps || !digits || rows < 0 || cols < 0 || ld < cols || nslices < 1 || nslices > DF_S_MAX)
    return DF_ERR_ARG;
  cudaError_t e = df::launch_split_rows_int8(A, rows, cols, ld, nslices, exps, digits, as_stream(stream));
  return e == cudaSuccess ? DF_OK : DF_ERR_CUDA;
}

}  // extern "C"

namespace {

// Shared driver of df_slice_products / df_emulated_gemm: split both operands
// into BF16 planes in scratch memory, run the slice GEMM, free the scratch.
df_status grid_gemm(const double *A, const double *B, int M, int N, int K, int s, int mode, int64_t *raw,
                    double *out, int32_t *ea_out, int32_t *eb_out, cudaStream_t st) {
  if (!A || !B || M <= 0 || N <= 0 || K <= 0 || s < 1 || s > DF_S_MAX) return DF_ERR_ARG;
  const long long ld = round_up(K, 8);
  // A B^T with B == A (a Gram matrix such as K_b = X_b X_b^T): one split serves both sides
  const bool same = A == B && M == N;
  uint16_t *Ad = nullptr, *Bd = nullptr;
  int *ea = nullptr, *eb = nullptr, *status = nullptr;
  df_status rs = DF_OK;
  cudaError_t e = df::scratch_malloc((void **)&Ad, sizeof(uint16_t) * (size_t)s * M * ld, st);
  if (e == cudaSuccess && !same) e = df::scratch_malloc((void **)&Bd, sizeof(uint16_t) * (size_t)s * N * ld, st);
  if (e == cudaSuccess) e = df::scratch_malloc((void **)&ea, sizeof(int) * M, st);
  if (e == cudaSuccess && !same) e = df::scratch_malloc((void **)&eb, sizeof(int) * N, st);
  if (e == cudaSuccess) e = df::scratch_malloc((void **)&status, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  // raw mode adds every chunk into its group's output: start from zero
  if (e == cudaSuccess && mode == df::kModeRaw) e = cudaMemsetAsync(raw, 0, sizeof(int64_t) * (size_t)s * M * N, st);
  if (e == cudaSuccess) e = df::launch_split_rows_bf16(A, M, K, K, s, ea, Ad, ld, (long long)M * ld, st);
  if (e == cudaSuccess && !same) e = df::launch_split_rows_bf16(B, N, K, K, s, eb, Bd, ld, (long long)N * ld, st);
  if (same) {
    Bd = Ad;
    eb = ea;
  }
  if (e == cudaSuccess) {
    CUtensorMap ta, tb;
    if (!df::make_tmap_bf16(&ta, Ad, K, M, s, ld, (long long)M * ld) ||
        !df::make_tmap_bf16(&tb, Bd, K, N, s, ld, (long long)N * ld)) {
      rs = DF_ERR_CUDA;
    } else {
      df::SgParams p;
      std::memset(&p, 0, sizeof(p));
      p.layout = df::kLayoutGrid;
      p.mode = mode;
      p.nt_m = (M + df::kTile - 1) / df::kTile;
      p.nt_n = (N + df::kTile - 1) / df::kTile;
      p.nunits = p.nt_m * p.nt_n;
      p.m_valid = M;
      p.n_valid = N;
      p.ktiles = (K + df::kKTile - 1) / df::kKTile;
      p.s_fixed = s;
      for (int q = 0; q <= 8; ++q) p.shiftT[q] = df::fixed_point_shift(q, (long long)p.ktiles * df::kKTile);
      p.ea = ea;
      p.eb = eb;
      p.out = out;
      p.out_ld = N;
      p.raw = reinterpret_cast<long long *>(raw);
      p.status = status;
      e = df::launch_slice_gemm(p, ta, tb, st);
    }
  }
  int h = 0;
  if (e == cudaSuccess && rs == DF_OK) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && rs == DF_OK && ea_out) e = cudaMemcpyAsync(ea_out, ea, sizeof(int) * M, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && rs == DF_OK && eb_out) e = cudaMemcpyAsync(eb_out, eb, sizeof(int) * N, cudaMemcpyDeviceToDevice, st);
  for (void *ptr : {(void *)Ad, same ? nullptr : (void *)Bd, (void *)ea, same ? nullptr : (void *)eb, (void *)status})
    if (ptr) cudaFreeAsync(ptr, st);
  cudaError_t es = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = es;
  if (rs != DF_OK) return rs;
  if (e != cudaSuccess) return DF_ERR_CUDA;
  return h ? DF_ERR_TIMEOUT : DF_OK;
}

}  // namespace

extern "C" {

df_status df_slice_products(const double *A, const double *B, int M, int N, int K, int nslices, int64_t *S,
                            int32_t *ea, int32_t *eb, void *stream) {
  if (!S) return DF_ERR_ARG;
  return grid_gemm(A, B, M, N, K, nslices, df::kModeRaw, S, nullptr, ea, eb, as_stream(stream));
}

df_status df_emulated_gemm(const double *A, const double *B, int M, int N, int K, int nslices, double *out,
                           void *stream) {
  if (!out) return DF_ERR_ARG;
  return grid_gemm(A, B, M, N, K, nslices, df::kModeGemm, nullptr, out, nullptr, nullptr, as_stream(stream));
}

}  // extern "C"
