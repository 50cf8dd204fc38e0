// Split kernels (Section 3.2): FP64 values -> one power-of-two exponent per
// row (or column) and balanced signed 8-bit digits, most significant first.
//
//   e      = smallest integer with max|row| < 127/128 * 2^e   (0 for a zero row)
//   N      = RNE(v * 2^(63-e))  (|N| < 127 * 2^56)
//   digits = seven balanced bytes from the bottom, the rest on top, so that
//            v 2^(63-e) = sum_t d_t 256^(7-t), d_t in [-128, 127], |d_0| <= 127.
//
// All of it is integer arithmetic on the FP64 bit patterns.  The digits feed
// the tensor cores as BF16 (every integer in [-256, 256] is exact in BF16).
// These kernels are HBM-bound: each reads its FP64 input once from DRAM (the
// second pass over a row hits L1/L2) and writes s bytes-worth of digits.
#include "df_internal.h"

namespace df {

namespace {

__device__ __forceinline__ uint64_t abs_bits(double v) {
  return (uint64_t)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// One warp per row; two columns per lane per step (16-byte loads, 4-byte stores).
__global__ void __launch_bounds__(256) split_rows_bf16_kernel(const double *__restrict__ A, long long rows,
                                                              int cols, long long ld, int nslices,
                                                              int *__restrict__ exps,
                                                              uint16_t *__restrict__ digits, long long dld,
                                                              long long plane_stride, int vec2,
                                                              const int *__restrict__ perm, int group) {
  const int lane = threadIdx.x & 31;
  const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  // with a permutation, output row r = (P', j) reads input row (perm[P'], j), `group` rows per P
  const long long src = perm ? (long long)perm[r / group] * group + (r % group) : r;
  const double *row = A + src * ld;
  uint64_t m = 0;
  if (vec2) {
    const double2 *row2 = reinterpret_cast<const double2 *>(row);
    const int half = cols >> 1;
    for (int c = lane; c < half; c += 32) {
      double2 v = __ldg(row2 + c);
      uint64_t a = abs_bits(v.x), b = abs_bits(v.y);
      m = a > m ? a : m;
      m = b > m ? b : m;
    }
    if ((cols & 1) && lane == 0) {
      uint64_t a = abs_bits(row[cols - 1]);
      m = a > m ? a : m;
    }
  } else {
    for (int c = lane; c < cols; c += 32) {
      uint64_t a = abs_bits(__ldg(row + c));
      m = a > m ? a : m;
    }
  }
  m = warp_max_u64(m);
  const int e = exponent_from_max_bits_dev(m);
  if (lane == 0) exps[r] = e;
  uint16_t *drow = digits + r * dld;
  for (int c = 2 * lane; c < cols; c += 64) {
    int d0[kSMax], d1[kSMax];
    uint64_t b0 = (uint64_t)__double_as_longlong(row[c]);
    balanced_digits(scaled_rne(b0, e), d0);
    bool two = c + 1 < cols;
    if (two) {
      uint64_t b1 = (uint64_t)__double_as_longlong(row[c + 1]);
      balanced_digits(scaled_rne(b1, e), d1);
    } else {
#pragma unroll
      for (int t = 0; t < kSMax; ++t) d1[t] = 0;
    }
#pragma unroll
    for (int t = 0; t < kSMax; ++t) {
      if (t < nslices) {
        uint32_t pk = (uint32_t)int_to_bf16_bits(d0[t]) | ((uint32_t)int_to_bf16_bits(d1[t]) << 16);
        uint16_t *dst = drow + (long long)t * plane_stride + c;
        if (two && ((reinterpret_cast<uintptr_t>(dst) & 3) == 0)) {
          *reinterpret_cast<uint32_t *>(dst) = pk;
        } else {
          dst[0] = (uint16_t)(pk & 0xFFFF);
          if (two) dst[1] = (uint16_t)(pk >> 16);
        }
      }
    }
  }
}

// One warp per row, int8 digits [nslices][rows][cols] (inspection entry point).
__global__ void split_rows_int8_kernel(const double *__restrict__ A, int rows, int cols, int ld, int nslices,
                                       int *__restrict__ exps, int8_t *__restrict__ digits) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const double *row = A + (long long)r * ld;
  uint64_t m = 0;
  for (int c = lane; c < cols; c += 32) {
    uint64_t a = abs_bits(row[c]);
    m = a > m ? a : m;
  }
  m = warp_max_u64(m);
  const int e = exponent_from_max_bits_dev(m);
  if (lane == 0) exps[r] = e;
  for (int c = lane; c < cols; c += 32) {
    int d[kSMax];
    balanced_digits(scaled_rne((uint64_t)__double_as_longlong(row[c]), e), d);
    for (int t = 0; t < nslices; ++t) digits[((long long)t * rows + r) * cols + c] = (int8_t)d[t];
  }
}

// One warp per column c of C [nrows][ncols]: digits go to [t][c][r] (K-major).
__global__ void split_cols_bf16_kernel(const double *__restrict__ C, int nrows, int ncols, int nslices,
                                       int *__restrict__ exps, uint16_t *__restrict__ digits, long long dld,
                                       long long plane_stride) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ncols) return;
  uint64_t m = 0;
  for (int r = lane; r < nrows; r += 32) {
    uint64_t a = abs_bits(C[(long long)r * ncols + c]);
    m = a > m ? a : m;
  }
  m = warp_max_u64(m);
  const int e = exponent_from_max_bits_dev(m);
  if (lane == 0) exps[c] = e;
  for (int r = lane; r < nrows; r += 32) {
    int d[kSMax];
    balanced_digits(scaled_rne((uint64_t)__double_as_longlong(C[(long long)r * ncols + c]), e), d);
    for (int t = 0; t < nslices; ++t)
      digits[(long long)t * plane_stride + (long long)c * dld + r] = int_to_bf16_bits(d[t]);
  }
}

// One CTA per (block b, row mu) of X [naux][nao][nocc]: the row of the second
// exchange GEMM is X_b[mu, (P_local, i)], length nP*nocc, padded with zero
// digits up to a multiple of 64, one exponent per (block, mu).  The first pass
// finds max|X| (from DRAM), the second re-reads the row (256 KB at most, from
// L2) and writes the digits.  Two consecutive orbitals per thread (16-byte
// loads, 4-byte stores) when nocc is even.
__global__ void __launch_bounds__(256) split_xblocks_kernel(const double *__restrict__ X, int naux, int nao,
                                                            int nocc, int nslices, int *__restrict__ eX,
                                                            uint16_t *__restrict__ Xd, long long kb_ld, int nblk) {
  const int mu = blockIdx.x;
  const int b = blockIdx.y;
  const int p0 = b * kBlock;
  const int nP = min(kBlock, naux - p0);
  const int klen = nP * nocc;
  const int kpad = (klen + 63) / 64 * 64;
  __shared__ uint64_t red[8];
  __shared__ int e_sh;
  {
    uint64_t m = 0;
    if ((nocc & 1) == 0) {
      const int hp = nocc >> 1;
      for (int q = threadIdx.x; q < nP * hp; q += blockDim.x) {
        const int pl = q / hp;
        const int i = 2 * (q - pl * hp);
        const double2 v = *reinterpret_cast<const double2 *>(X + ((long long)(p0 + pl) * nao + mu) * nocc + i);
        const uint64_t a = abs_bits(v.x), c = abs_bits(v.y);
        m = a > m ? a : m;
        m = c > m ? c : m;
      }
    } else {
      for (int k = threadIdx.x; k < klen; k += blockDim.x) {
        const int pl = k / nocc;
        const uint64_t a = abs_bits(X[((long long)(p0 + pl) * nao + mu) * nocc + (k - pl * nocc)]);
        m = a > m ? a : m;
      }
    }
    m = warp_max_u64(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint64_t v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
      v = warp_max_u64(v);
      if (threadIdx.x == 0) {
        e_sh = exponent_from_max_bits_dev(v);
        eX[b * nao + mu] = e_sh;
      }
    }
    __syncthreads();
  }
  const int e = e_sh;
  const long long plane = (long long)nblk * nao * kb_ld;
  uint16_t *dst = Xd + ((long long)b * nao + mu) * kb_ld;
  if ((nocc & 1) == 0) {
    const int hp = nocc >> 1;
    for (int q = threadIdx.x; 2 * q < kpad; q += blockDim.x) {
      const int k = 2 * q;
      int d0[kSMax], d1[kSMax];
      if (k < klen) {
        const int pl = q / hp;
        const int i = k - pl * nocc;
        const double2 v = *reinterpret_cast<const double2 *>(X + ((long long)(p0 + pl) * nao + mu) * nocc + i);
        balanced_digits(scaled_rne((uint64_t)__double_as_longlong(v.x), e), d0);
        balanced_digits(scaled_rne((uint64_t)__double_as_longlong(v.y), e), d1);
      } else {
#pragma unroll
        for (int t = 0; t < kSMax; ++t) d0[t] = d1[t] = 0;
      }
#pragma unroll
      for (int t = 0; t < kSMax; ++t)
        if (t < nslices)
          *reinterpret_cast<uint32_t *>(dst + (long long)t * plane + k) =
              (uint32_t)int_to_bf16_bits(d0[t]) | ((uint32_t)int_to_bf16_bits(d1[t]) << 16);
    }
  } else {
    for (int k = threadIdx.x; k < kpad; k += blockDim.x) {
      int d[kSMax];
      if (k < klen) {
        const int pl = k / nocc;
        const int i = k - pl * nocc;
        balanced_digits(scaled_rne((uint64_t)__double_as_longlong(X[((long long)(p0 + pl) * nao + mu) * nocc + i]), e),
                        d);
      } else {
#pragma unroll
        for (int t = 0; t < kSMax; ++t) d[t] = 0;
      }
#pragma unroll
      for (int t = 0; t < kSMax; ++t)
        if (t < nslices) dst[(long long)t * plane + k] = int_to_bf16_bits(d[t]);
    }
  }
}

// K[mu][nu] = sum_b fl( 2^(eX[b,mu] + eX[b,nu] - 14 - 8(s_b - 1) + T(s_b)) * sum_sp R[b,sp] ),
// blocks in order (FP64), where R[b,sp][hi][lo] are the exact int64 partials of
// the second exchange GEMM (lower block-triangle, transposed) and the sum over
// the K splits of a block is exact.
__global__ void kpart_reduce_kernel(const long long *__restrict__ Rp, const int *__restrict__ eX,
                                    const int *__restrict__ s_blk, ShiftTable shiftT, int nao, int nblk, int nsplit,
                                    double *__restrict__ K) {
  const int nu = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (nu >= nao) return;
  const int hi = mu > nu ? mu : nu;
  const int lo = mu > nu ? nu : mu;
  const long long off = (long long)hi * nao + lo;
  const long long bs = (long long)nao * nao;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) {
    long long R = 0;
    for (int sp = 0; sp < nsplit; ++sp) R += Rp[((long long)b * nsplit + sp) * bs + off];
    const int s = s_blk[b];
    const int k = eX[b * nao + mu] + eX[b * nao + nu] - 14 - 8 * (s - 1) + shiftT.v[s];
    acc += ldexp_i64(R, k);
  }
  K[(long long)mu * nao + nu] = acc;
}

}  // namespace

cudaError_t launch_split_rows_bf16(const double *A, long long rows, int cols, long long ld, int nslices,
                                   int *exps, uint16_t *digits, long long dld, long long plane_stride,
                                   cudaStream_t st, const int *perm, int group) {
  if (rows <= 0) return cudaSuccess;
  const int vec2 = ((ld & 1) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0) ? 1 : 0;
  const int wpb = 8;
  dim3 grid((unsigned)((rows + wpb - 1) / wpb));
  split_rows_bf16_kernel<<<grid, 32 * wpb, 0, st>>>(A, rows, cols, ld, nslices, exps, digits, dld,
                                                    plane_stride, vec2, perm, group > 0 ? group : 1);
  return cudaGetLastError();
}

cudaError_t launch_split_rows_int8(const double *A, int rows, int cols, int ld, int nslices, int *exps,
                                   int8_t *digits, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  split_rows_int8_kernel<<<(rows + 7) / 8, 256, 0, st>>>(A, rows, cols, ld, nslices, exps, digits);
  return cudaGetLastError();
}

cudaError_t launch_split_cols_bf16(const double *C, int nrows, int ncols, int nslices, int *exps,
                                   uint16_t *digits, long long dld, long long plane_stride, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  split_cols_bf16_kernel<<<(ncols + 7) / 8, 256, 0, st>>>(C, nrows, ncols, nslices, exps, digits, dld,
                                                          plane_stride);
  return cudaGetLastError();
}

cudaError_t launch_split_xblocks(const double *X, int naux, int nao, int nocc, int nslices, int *eX, uint16_t *Xd,
                                 long long kb_ld, int nblk, cudaStream_t st) {
  dim3 grid(nao, nblk);
  split_xblocks_kernel<<<grid, 256, 0, st>>>(X, naux, nao, nocc, nslices, eX, Xd, kb_ld, nblk);
  return cudaGetLastError();
}

cudaError_t launch_kpart_reduce(const long long *Rp, const int *eX, const int *s_blk, ShiftTable shiftT, int nao,
                                int nblk, int nsplit, double *K, cudaStream_t st) {
  dim3 grid((nao + 127) / 128, nao);
  kpart_reduce_kernel<<<grid, 128, 0, st>>>(Rp, eX, s_blk, shiftT, nao, nblk, nsplit, K);
  return cudaGetLastError();
}

}  // namespace df
