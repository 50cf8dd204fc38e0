// Coulomb build in FP64 (Section 2.1, Eqs. df-j-1 and df-j-2) and the energy
// reductions.
//
//   rho_P = sum_mn B_Pmn D_mn     (one streaming pass over B)
//   J_mn  = sum_P B_Pmn rho_P     (a second streaming pass over B)
//
// Both B_P and D are symmetric (D by the paper's assumption in Section 2.1,
// B_P by construction), so each pass reads only the upper triangle of every
// B_P: nao(nao+1)/2 doubles per auxiliary function instead of nao^2.  That
// halves the DRAM bytes and the FP64 FMAs of the paper's 4 N_scr N_aux
// (Section 3.1).  On GB300 the FP64 pipe is narrow, so these kernels are
// bounded by FP64 FMA throughput rather than by HBM; the roofline reported
// for them uses the measured FP64 rate.
//
// B comes dense ([naux][nao][nao]) or packed (per P the upper triangle row by
// row, [naux][nao (nao + 1) / 2], the symmetric storage Section 3.3
// describes); both layouts are read in the same order, so rho and J are
// bit-identical between them.
//
// A Schwarz-screened B (Section 2.1: a screened AO pair is zero in every B_P)
// is block-sparse: with per-mu masks of the 64-wide nu chunks that hold a
// nonzero, both passes skip the zero chunks (rho loses only zero terms; J is
// exactly zero there), cutting bytes and FMAs to the surviving pairs.
#include "df_internal.h"

namespace df {

namespace {

// Start of row mu in a packed upper triangle of order nao.
__device__ __forceinline__ long long packed_row(int mu, int nao) {
  return (long long)mu * nao - (long long)mu * (mu - 1) / 2;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Work items of a launch: with a null counter the CTA takes its own index
// once; otherwise the CTAs of a short grid (a few per SM, sharing the SMs
// with another kernel) take items from the counter until they run out.  The
// value is uniform over the CTA.
__device__ __forceinline__ int take_item(int *work, int *slot) {
  if (threadIdx.x == 0) *slot = atomicAdd(work, 1);
  __syncthreads();
  const int v = *slot;
  __syncthreads();
  return v;
}

// The strictly upper elements of B_P in row-pair order: pair q < nao/2 is
// row q from nu = q + 1 followed by row nao-1-q from nu = nao-q (nao - 1
// elements together, so every pair has the same length); for odd nao the
// middle row, q = nao/2, comes last alone.  Thread t of the CTA takes the
// elements t, t + 256, t + 512, ...: each warp reads 32 consecutive values of
// one row, and no thread has a per-row tail.
struct PairStream {
  int q, e;       // the current element: offset e in pair q
  int nao, L;     // L = nao - 1, the length of a full pair
  __device__ __forceinline__ void init(int j0, int n) {
    nao = n;
    L = n - 1;
    q = j0 / L;
    e = j0 - q * L;
  }
  __device__ __forceinline__ bool valid() const {
    return 2 * q + 1 < nao || (2 * q + 1 == nao && e < nao - 1 - q);
  }
  // (mu, nu), nu > mu, of the current element
  __device__ __forceinline__ void at(int &mu, int &nu) const {
    if (e < nao - 1 - q) {
      mu = q;
      nu = q + 1 + e;
    } else {
      mu = nao - 1 - q;
      nu = e + 1;
    }
  }
  __device__ __forceinline__ void advance(int step) {
    e += step;
    while (e >= L) {
      e -= L;
      ++q;
    }
  }
};

// rho_P for one P by one CTA of 256 threads:
//   rho_P = sum_mu B_P mu mu D_mu mu + 2 sum_{mu < nu} B_P mu nu D_mu nu.
// The diagonal terms are spread over the threads; the strictly upper ones
// stream in row-pair order (PairStream), eight loads ahead of their FMAs (a
// ring of registers, FMAs in stream order), so that a few CTAs per SM keep
// enough bytes in flight to share the SM with another kernel.
template <bool kPacked>
__device__ __forceinline__ void rho_one(const double *__restrict__ B, const double *__restrict__ D, int nao,
                                        double *__restrict__ rho, int P, double *red) {
  constexpr int kQ = 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double *BP = B + (long long)P * (kPacked ? (long long)nao * (nao + 1) / 2 : (long long)nao * nao);
  auto badr = [&](int mu, int nu) -> const double * {
    return kPacked ? BP + packed_row(mu, nao) + (nu - mu) : BP + (long long)mu * nao + nu;
  };
  double dia = 0.0;
  for (int mu = tid; mu < nao; mu += 256) dia = fma(__ldg(badr(mu, mu)), __ldg(D + (long long)mu * nao + mu), dia);
  double off = 0.0;
  const long long total = (long long)nao * (nao - 1) / 2;
  if (total > tid) {
    PairStream ps;
    ps.init(tid, nao);
    double bq[kQ], dq[kQ];
    auto fill = [&](int k) {
      bq[k] = 0.0;
      dq[k] = 0.0;
      if (ps.valid()) {
        int mu, nu;
        ps.at(mu, nu);
        bq[k] = __ldg(badr(mu, nu));
        dq[k] = __ldg(D + (long long)mu * nao + nu);
      }
      ps.advance(256);
    };
#pragma unroll
    for (int k = 0; k < kQ; ++k) fill(k);
    const long long mine = (total - tid + 255) / 256;
    const int rounds = (int)((mine + kQ - 1) / kQ);
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
      for (int k = 0; k < kQ; ++k) {
        off = fma(bq[k], dq[k], off);
        fill(k);
      }
    }
  }
  double v = 2.0 * off + dia;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    rho[P] = t;
  }
  __syncthreads();
}

// rho_P for a B with zero 64-wide chunks (a Schwarz-screened B), row by row:
// warp w takes rows mu = w, w + 8, ...; lanes stride nu > mu.  With masks a
// warp skips each 32-wide window whose chunks are all zero as a whole (no
// loads, no FMAs) and keeps the order of the rest; without (DF_OPT_SPARSE
// off) it runs every window in the same order, so the two are bit-identical
// (a skipped term is an exact zero).  The row-pair stream would visit every
// element of the triangle to skip the zero ones.
template <bool kPacked>
__device__ __forceinline__ void rho_one_rows(const double *__restrict__ B, const double *__restrict__ D, int nao,
                                             double *__restrict__ rho, const uint32_t *__restrict__ mask_mu, int P,
                                             double *red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double *BP = B + (long long)P * (kPacked ? (long long)nao * (nao + 1) / 2 : (long long)nao * nao);
  double off = 0.0, dia = 0.0;
  for (int mu = warp; mu < nao; mu += 8) {
    // brow[nu] is B_P mu nu for nu >= mu in either layout
    const double *brow = kPacked ? BP + packed_row(mu, nao) - mu : BP + (long long)mu * nao;
    const double *drow = D + (long long)mu * nao;
    if (lane == 0) dia = fma(__ldg(brow + mu), __ldg(drow + mu), dia);
    if (!mask_mu) {
      for (int nu = mu + 1 + lane; nu < nao; nu += 32) off = fma(__ldg(brow + nu), __ldg(drow + nu), off);
    } else {
      const uint32_t mk = __ldg(mask_mu + mu);
      for (int base = mu + 1; base < nao; base += 32) {
        if (!(((mk >> (base >> 6)) | (mk >> ((base + 31) >> 6))) & 1u)) continue;
        const int nu = base + lane;
        if (nu < nao && ((mk >> (nu >> 6)) & 1u)) off = fma(__ldg(brow + nu), __ldg(drow + nu), off);
      }
    }
  }
  double v = 2.0 * off + dia;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    rho[P] = t;
  }
  __syncthreads();
}

// One CTA per P (work == null), or a short grid taking P from the counter.
// kRows: the row-by-row order of a B with zero chunks (masks optional).  At
// most 48 registers, like the J kernel.
template <bool kPacked, bool kRows>
__global__ void __launch_bounds__(256, 5) rho_kernel(const double *__restrict__ B, const double *__restrict__ D,
                                                     int naux, int nao, double *__restrict__ rho,
                                                     const uint32_t *__restrict__ mask_mu, int *__restrict__ work) {
  __shared__ double red[8];
  __shared__ int slot;
  if (!work) {
    if (kRows)
      rho_one_rows<kPacked>(B, D, nao, rho, mask_mu, blockIdx.x, red);
    else
      rho_one<kPacked>(B, D, nao, rho, blockIdx.x, red);
    return;
  }
  for (;;) {
    const int P = take_item(work, &slot);
    if (P >= naux) break;
    if (kRows)
      rho_one_rows<kPacked>(B, D, nao, rho, mask_mu, P, red);
    else
      rho_one<kPacked>(B, D, nao, rho, P, red);
  }
}

// J_mn = sum_P B_Pmn rho_P over the upper triangle, written to both halves.
// Item (x, y) takes elements x*256 .. of the row pair (y, nao-1-y): row y from
// column y, then row nao-1-y from its diagonal (nao + 1 elements per pair, one
// row alone in the middle when nao is odd), so every item has the same work.
// Each element's sum runs over P in ascending order, one FMA per P, with
// eight loads of B ahead of their FMAs.
template <bool kPacked>
__device__ __forceinline__ void coulomb_one(const double *__restrict__ B, const double *srho, int naux, int nao,
                                            double *__restrict__ J, const uint32_t *__restrict__ mask_mu, int x,
                                            int y) {
  const int m0 = y, m1 = nao - 1 - m0;
  const int len0 = nao - m0, len1 = m1 > m0 ? nao - m1 : 0;
  const int e = x * blockDim.x + threadIdx.x;
  if (e >= len0 + len1) return;
  const int mu = e < len0 ? m0 : m1;
  const int nu = e < len0 ? m0 + e : m1 + (e - len0);
  const long long off = kPacked ? packed_row(mu, nao) + (nu - mu) : (long long)mu * nao + nu;
  const long long stride = kPacked ? (long long)nao * (nao + 1) / 2 : (long long)nao * nao;
  const long long jmn = (long long)mu * nao + nu;
  if (mask_mu && !((__ldg(mask_mu + mu) >> (nu >> 6)) & 1u)) {
    // a screened pair: B_P mu nu = 0 for every P
    J[jmn] = 0.0;
    J[(long long)nu * nao + mu] = 0.0;
    return;
  }
  const double *bp = B + off;
  double acc = 0.0;
  int P = 0;
  for (; P + 8 <= naux; P += 8) {
    double b[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) b[q] = __ldg(bp + (P + q) * stride);
#pragma unroll
    for (int q = 0; q < 8; ++q) acc = fma(b[q], srho[P + q], acc);
  }
  for (; P < naux; ++P) acc = fma(__ldg(bp + P * stride), srho[P], acc);
  J[jmn] = acc;
  J[(long long)nu * nao + mu] = acc;
}

// Grid (gx, gy) of items (work == null), or a short grid taking item
// x + gx y from the counter.  At most 48 registers, so that a short grid of a
// few CTAs per SM leaves room for the X split's CTAs.
template <bool kPacked>
__global__ void __launch_bounds__(256, 5) coulomb_kernel(const double *__restrict__ B,
                                                         const double *__restrict__ rho, int naux, int nao,
                                                         double *__restrict__ J,
                                                         const uint32_t *__restrict__ mask_mu,
                                                         int *__restrict__ work, int gx, int nitems) {
  extern __shared__ double srho[];
  __shared__ int slot;
  for (int i = threadIdx.x; i < naux; i += blockDim.x) srho[i] = rho[i];
  __syncthreads();
  if (!work) {
    coulomb_one<kPacked>(B, srho, naux, nao, J, mask_mu, blockIdx.x, blockIdx.y);
    return;
  }
  for (;;) {
    const int it = take_item(work, &slot);
    if (it >= nitems) break;
    coulomb_one<kPacked>(B, srho, naux, nao, J, mask_mu, it % gx, it / gx);
  }
}

// Partial sums: [0] sum D.J, [1] sum rho.rho, [2] sum D.K, one triple per block.
__global__ void __launch_bounds__(256) energy_partials_kernel(const double *__restrict__ D,
                                                              const double *__restrict__ J,
                                                              const double *__restrict__ K,
                                                              const double *__restrict__ rho, long long n2,
                                                              int naux, double *__restrict__ part) {
  double a = 0.0, b = 0.0, c = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    const double d = D[i];
    if (J) a = fma(d, J[i], a);
    if (K) c = fma(d, K[i], c);
  }
  if (rho)
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < naux; i += stride)
      b = fma(rho[i], rho[i], b);
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  __shared__ double red[3][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][warp] = a;
    red[1][warp] = b;
    red[2][warp] = c;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
    part[blockIdx.x * 3 + threadIdx.x] = s;
  }
}

__global__ void energy_final_kernel(const double *__restrict__ part, int nblocks, double *__restrict__ E) {
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = 0; i < nblocks; ++i) {
      a += part[3 * i];
      b += part[3 * i + 1];
      c += part[3 * i + 2];
    }
    E[0] = 0.5 * a;
    E[1] = 0.5 * b;
    E[2] = -0.5 * c;
  }
}

// Partial sums of (D - D_prev)^2 per block; D_prev == nullptr: no previous density.
__global__ void __launch_bounds__(256) density_change_kernel(const double *__restrict__ D,
                                                             const double *__restrict__ Dprev, long long n2,
                                                             double *__restrict__ part) {
  double a = 0.0;
  if (Dprev) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
      const double d = D[i] - Dprev[i];
      a = fma(d, d, a);
    }
  }
  a = warp_sum(a);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

// ||D - D_prev||_F from the partials, or 1 when there is no previous density.
__global__ void density_change_final_kernel(const double *__restrict__ part, int nblocks, bool have_prev,
                                            double *__restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nblocks; ++i) s += part[i];
    *out = have_prev ? sqrt(s) : 1.0;
  }
}

// Sets *flag when some B_P is not exactly symmetric (a NaN counts as
// asymmetric).  Block (x, y, P) with x <= y compares the 32 x 32 tile (x, y) of
// B_P, staged in shared memory, with the transpose of tile (y, x).
__global__ void __launch_bounds__(256) symmetry_check_kernel(const double *__restrict__ B, int nao,
                                                             int *__restrict__ flag) {
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bi > bj) return;
  __shared__ double t[32][33];
  const double *BP = B + (long long)blockIdx.z * nao * nao;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + tx;
    if (i < nao && j < nao) t[r][tx] = BP[(long long)i * nao + j];
  }
  __syncthreads();
  bool bad = false;
  for (int r = ty; r < 32; r += 8) {
    const int i = bj * 32 + r, j = bi * 32 + tx;  // B[i][j] must equal B[j][i] = t[tx][r]
    if (i < nao && j < nao && !(BP[(long long)i * nao + j] == t[tx][r])) bad = true;
  }
  if (__any_sync(0xffffffffu, bad) && tx == 0) atomicOr(flag, 1);
}

// Per mu: bit c set when some B_P mu nu, nu in [64c, 64c + 64), is nonzero.
// One CTA per mu, over every P (one pass over B at setup).
__global__ void __launch_bounds__(256) pair_mask_kernel(const double *__restrict__ B, int naux, int nao,
                                                        uint32_t *__restrict__ mask_mu) {
  const int mu = blockIdx.x;
  uint32_t bits = 0u;
  const long long n2 = (long long)nao * nao;
  for (int P = 0; P < naux; ++P) {
    const double *row = B + (long long)P * n2 + (long long)mu * nao;
    for (int nu = threadIdx.x; nu < nao; nu += blockDim.x)
      if (__ldg(row + nu) != 0.0) bits |= 1u << (nu >> 6);
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  __shared__ uint32_t red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bits;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) bits |= red[w];
    mask_mu[mu] = bits;
  }
}

// Packed B: flag[k] = 1 when the packed pair k (of the upper triangle) is
// nonzero in some B_P (one coalesced pass over B), then the per-mu masks
// over all nu from the symmetric pair flags.
__global__ void __launch_bounds__(256) packed_pair_flags_kernel(const double *__restrict__ Bp, int naux,
                                                                long long npk, uint8_t *__restrict__ flag) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npk) return;
  uint8_t f = 0;
  for (int P = 0; P < naux && !f; ++P) f = __ldg(Bp + (long long)P * npk + k) != 0.0;
  flag[k] = f;
}

__global__ void mask_from_packed_flags_kernel(const uint8_t *__restrict__ flag, int nao,
                                              uint32_t *__restrict__ mask_mu) {
  const int mu = blockIdx.x * blockDim.x + threadIdx.x;
  if (mu >= nao) return;
  uint32_t bits = 0u;
  for (int nu = 0; nu < nao; ++nu) {
    const long long k = nu >= mu ? packed_row(mu, nao) + (nu - mu) : packed_row(nu, nao) + (mu - nu);
    if (flag[k]) bits |= 1u << (nu >> 6);
  }
  mask_mu[mu] = bits;
}

// Dense copy of B_P for P = P0 .. P0 + nP - 1 from the packed layout.
__global__ void unpack_kernel(const double *__restrict__ Bp, int P0, int nP, int nao, double *__restrict__ out) {
  const long long npk = (long long)nao * (nao + 1) / 2;
  const long long n2 = (long long)nao * nao;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nP * n2) return;
  const int pl = (int)(i / n2);
  const int mu = (int)((i - pl * n2) / nao), nu = (int)(i - pl * n2 - (long long)mu * nao);
  const int lo = mu < nu ? mu : nu, hi = mu < nu ? nu : mu;
  out[i] = __ldg(Bp + (long long)(P0 + pl) * npk + packed_row(lo, nao) + (hi - lo));
}

// Per 128-row tile t of the (P, mu) rows (row r has mu = r mod nao): the OR of
// its rows' masks.
__global__ void tile_mask_kernel(const uint32_t *__restrict__ mask_mu, int nao, long long rows, int ntiles,
                                 uint32_t *__restrict__ mask_tile) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  uint32_t m = 0u;
  const long long r0 = (long long)t * kTile;
  for (long long r = r0; r < r0 + kTile && r < rows; ++r) m |= mask_mu[r % nao];
  mask_tile[t] = m;
}

}  // namespace

constexpr int kEnergyBlocks = 296;

cudaError_t launch_pair_masks_packed(const double *Bp, int naux, int nao, uint32_t *mask_mu, uint32_t *mask_tile,
                                     cudaStream_t st) {
  const long long npk = (long long)nao * (nao + 1) / 2;
  uint8_t *flag = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&flag), (size_t)npk, st);
  if (e != cudaSuccess) return e;
  packed_pair_flags_kernel<<<(unsigned)((npk + 255) / 256), 256, 0, st>>>(Bp, naux, npk, flag);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    mask_from_packed_flags_kernel<<<(nao + 127) / 128, 128, 0, st>>>(flag, nao, mask_mu);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const long long rows = (long long)naux * nao;
    const int ntiles = (int)((rows + kTile - 1) / kTile);
    tile_mask_kernel<<<(ntiles + 255) / 256, 256, 0, st>>>(mask_mu, nao, rows, ntiles, mask_tile);
    e = cudaGetLastError();
  }
  cudaFreeAsync(flag, st);
  return e;
}

cudaError_t launch_unpack(const double *Bp, int P0, int nP, int nao, double *out, cudaStream_t st) {
  const long long n = (long long)nP * nao * nao;
  unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Bp, P0, nP, nao, out);
  return cudaGetLastError();
}

cudaError_t launch_symmetry_check(const double *B, int naux, int nao, int *flag, cudaStream_t st) {
  const int nt = (nao + 31) / 32;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  for (int p0 = 0; p0 < naux; p0 += 65535) {
    const int np = naux - p0 < 65535 ? naux - p0 : 65535;
    symmetry_check_kernel<<<dim3(nt, nt, np), 256, 0, st>>>(B + (long long)p0 * nao * nao, nao, flag);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_pair_masks(const double *B, int naux, int nao, uint32_t *mask_mu, uint32_t *mask_tile,
                              cudaStream_t st) {
  pair_mask_kernel<<<nao, 256, 0, st>>>(B, naux, nao, mask_mu);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long rows = (long long)naux * nao;
  const int ntiles = (int)((rows + kTile - 1) / kTile);
  tile_mask_kernel<<<(ntiles + 255) / 256, 256, 0, st>>>(mask_mu, nao, rows, ntiles, mask_tile);
  return cudaGetLastError();
}

cudaError_t launch_density_change(const double *D, double *Dprev, bool have_prev, long long n2, double *part,
                                  double *out, cudaStream_t st) {
  density_change_kernel<<<kDensityChangeBlocks, 256, 0, st>>>(D, have_prev ? Dprev : nullptr, n2, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  density_change_final_kernel<<<1, 32, 0, st>>>(part, kDensityChangeBlocks, have_prev, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(Dprev, D, sizeof(double) * n2, cudaMemcpyDeviceToDevice, st);
}

cudaError_t launch_rho(const double *B, const double *D, int naux, int nao, double *rho, cudaStream_t st,
                       const uint32_t *mask_mu, bool packed, int *work, int grid, bool rows) {
  const unsigned g = work ? (unsigned)grid : (unsigned)naux;
  rows = rows || mask_mu;
  if (packed) {
    if (rows)
      rho_kernel<true, true><<<g, 256, 0, st>>>(B, D, naux, nao, rho, mask_mu, work);
    else
      rho_kernel<true, false><<<g, 256, 0, st>>>(B, D, naux, nao, rho, nullptr, work);
  } else {
    if (rows)
      rho_kernel<false, true><<<g, 256, 0, st>>>(B, D, naux, nao, rho, mask_mu, work);
    else
      rho_kernel<false, false><<<g, 256, 0, st>>>(B, D, naux, nao, rho, nullptr, work);
  }
  return cudaGetLastError();
}

cudaError_t launch_coulomb(const double *B, const double *rho, int naux, int nao, double *J, cudaStream_t st,
                           const uint32_t *mask_mu, bool packed, int *work, int grid) {
  const size_t sm = (size_t)naux * sizeof(double);
  static size_t attr = 48 * 1024;
  if (sm > attr) {
    cudaError_t e = cudaFuncSetAttribute(coulomb_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(coulomb_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = sm;
  }
  const int gx = (nao + 1 + 255) / 256, gy = (nao + 1) / 2;
  const dim3 g = work ? dim3((unsigned)grid) : dim3(gx, gy);
  if (packed)
    coulomb_kernel<true><<<g, 256, sm, st>>>(B, rho, naux, nao, J, mask_mu, work, gx, gx * gy);
  else
    coulomb_kernel<false><<<g, 256, sm, st>>>(B, rho, naux, nao, J, mask_mu, work, gx, gx * gy);
  return cudaGetLastError();
}

cudaError_t launch_energy(const double *D, const double *J, const double *K, const double *rho, int nao, int naux,
                          double *partials, double *E_dev, cudaStream_t st) {
  energy_partials_kernel<<<kEnergyBlocks, 256, 0, st>>>(D, J, K, rho, (long long)nao * nao, naux, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  energy_final_kernel<<<1, 32, 0, st>>>(partials, kEnergyBlocks, E_dev);
  return cudaGetLastError();
}

}  // namespace df
