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
// These kernels are HBM-bound: each reads its FP64 input and writes s
// digits per value, in two passes over a row (its maximum, then the digits);
// for the B and C splits the second pass mostly hits L1/L2.  The X split's
// rows (128 functions x nocc values, up to 256 KB) take their exponent bound
// from the first GEMM and are read once.
#include "df_internal.h"

#include <climits>
#include <type_traits>

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

// Largest absolute bit pattern over the TPR threads of a row (TPR = 32: one
// warp; TPR = 256: the whole block, through shared memory).
template <int TPR>
__device__ __forceinline__ uint64_t row_max_u64(uint64_t m) {
  m = warp_max_u64(m);
  if (TPR > 32) {
    __shared__ uint64_t part[TPR / 32];
    const int w = (threadIdx.x & (TPR - 1)) >> 5;
    if ((threadIdx.x & 31) == 0) part[w] = m;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TPR / 32; ++i) m = part[i] > m ? part[i] : m;
  }
  return m;
}

// TPR threads per row (a warp, or the whole block for wide rows so that a
// few hundred rows of tens of thousands of columns still fill the GPU); two
// columns per thread per step (16-byte loads, 4-byte stores).
template <int TPR>
__global__ void __launch_bounds__(256) split_rows_bf16_kernel(const double *__restrict__ A, long long rows,
                                                              int cols, long long ld, int nslices,
                                                              int *__restrict__ exps,
                                                              uint16_t *__restrict__ digits, long long dld,
                                                              long long plane_stride, int vec2,
                                                              const int *__restrict__ perm, int group) {
  const int lane = threadIdx.x & (TPR - 1);
  const long long r = (long long)blockIdx.x * (blockDim.x / TPR) + (threadIdx.x / TPR);
  if (r >= rows) return;  // uniform over a row's threads (a whole block when TPR = 256)
  // with a permutation, output row r = (P', j) reads input row (perm[P'], j), `group` rows per P
  const long long src = perm ? (long long)perm[r / group] * group + (r % group) : r;
  const double *row = A + src * ld;
  uint64_t m = 0;
  if (vec2) {
    const double2 *row2 = reinterpret_cast<const double2 *>(row);
    const int half = cols >> 1;
    for (int c = lane; c < half; c += TPR) {
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
    for (int c = lane; c < cols; c += TPR) {
      uint64_t a = abs_bits(__ldg(row + c));
      m = a > m ? a : m;
    }
  }
  m = row_max_u64<TPR>(m);
  const int e = exponent_from_max_bits_dev(m);
  if (lane == 0) exps[r] = e;
  uint16_t *drow = digits + r * dld;
  for (int c = 2 * lane; c < cols; c += 2 * TPR) {
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

// Rows of B from its packed layout (per P the upper triangle row by row,
// nao (nao + 1) / 2 values): output row r = (P', mu), P = perm[P'] (or P'),
// holds B_P mu nu for every nu (nu < mu read at the transposed position).
// One warp per row; the same two passes and digits as split_rows_bf16_kernel.
__global__ void __launch_bounds__(256) split_rows_packed_kernel(const double *__restrict__ Bp, long long rows,
                                                                int nao, int nslices, int *__restrict__ exps,
                                                                uint16_t *__restrict__ digits, long long dld,
                                                                long long plane_stride,
                                                                const int *__restrict__ perm) {
  const int lane = threadIdx.x & 31;
  const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const int Pq = (int)(r / nao), mu = (int)(r - (long long)Pq * nao);
  const int P = perm ? perm[Pq] : Pq;
  const double *BP = Bp + (long long)P * ((long long)nao * (nao + 1) / 2);
  const long long row_mu = (long long)mu * nao - (long long)mu * (mu - 1) / 2 - mu;  // + nu for nu >= mu
  auto at = [&](int nu) -> double {
    return nu >= mu ? __ldg(BP + row_mu + nu)
                    : __ldg(BP + (long long)nu * nao - (long long)nu * (nu - 1) / 2 + (mu - nu));
  };
  uint64_t m = 0;
  for (int c = lane; c < nao; c += 32) {
    const uint64_t a = abs_bits(at(c));
    m = a > m ? a : m;
  }
  m = warp_max_u64(m);
  const int e = exponent_from_max_bits_dev(m);
  if (lane == 0) exps[r] = e;
  uint16_t *drow = digits + r * dld;
  for (int c = 2 * lane; c < nao; c += 64) {
    int d0[kSMax], d1[kSMax];
    balanced_digits(scaled_rne((uint64_t)__double_as_longlong(at(c)), e), d0);
    const bool two = c + 1 < nao;
    if (two) {
      balanced_digits(scaled_rne((uint64_t)__double_as_longlong(at(c + 1)), e), d1);
    } else {
#pragma unroll
      for (int t = 0; t < kSMax; ++t) d1[t] = 0;
    }
#pragma unroll
    for (int t = 0; t < kSMax; ++t) {
      if (t < nslices) {
        const uint32_t pk = (uint32_t)int_to_bf16_bits(d0[t]) | ((uint32_t)int_to_bf16_bits(d1[t]) << 16);
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
// digits up to a multiple of 64, one exponent per (block, mu).
//
// The first exchange GEMM leaves X as its exact int64 fixed-point sums R
// (Section 3.2's recombination before the final rounding); this kernel takes
// X = fl64(R 2^k), k = -14 - 8(s_b - 1) + T(s_b) + eC[i] + eB[(P, mu)], the
// one rounding of the emulated product, and splits it.  (Doing the rounding
// here keeps the GEMM's epilogue short; it measured 18% faster that way.)
// The row's exponent needs its largest |X| (exact magnitude keys).  When the
// first GEMM recorded its bound E for the row (rowE), the exponent is E or
// E + 1, so one pass writes the digits with E while it takes the keys, and
// only a row whose exact exponent differs (about one in a hundred) is read
// a second time; R is read once.  Without the bound, a first pass takes the
// keys and a second re-reads the row (256 KB at most, mostly from DRAM) for
// the digits.  Two consecutive orbitals per thread (16-byte loads, 4-byte
// stores) when nocc is even.
template <int M>
using Mode = std::integral_constant<int, M>;  // digits_pass: 0 digits, 1 and keys, 2 and threshold bits

constexpr int kSplitXThreads = 256;
constexpr int kSplitXMinBlocks = 6;  // 40 registers: six rows in flight per SM (four at 51 measured slower)
constexpr int kP1 = 4;  // loads in flight per thread in the first pass (8 measured slower)

// Digit t of the balanced expansion of N as an exact FP32 value, from
// M = N + 128 (1 + 256 + ... + 256^6): the top digit is M >> 56, digit t >= 1
// is byte 7-t of M minus 128.  The FP32 is built as (1.5 2^23 + byte) - (1.5
// 2^23 + 128): one byte permute places the byte under the exponent bits and
// one FP32 subtraction is exact, so its top 16 bits are the digit's BF16.
__device__ __forceinline__ float digit_f32(long long M, int t) {
  if (t == 0) return __int_as_float(0x4B400000 + (int)(M >> 56)) - 12582912.0f;
  const uint32_t w = (7 - t) >= 4 ? (uint32_t)((unsigned long long)M >> 32) : (uint32_t)M;
  return __int_as_float((int)__byte_perm(w, 0x4B400000u, 0x7640u | (uint32_t)((7 - t) & 3))) - 12583040.0f;
}

// BF16 of two FP32 digits (exact) packed low, high.
__device__ __forceinline__ uint32_t bf16x2_of(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632u);
}

struct XScale {
  const int *eB, *eC;  // (P, mu) row and orbital exponents of the first GEMM
  const int *s_blk;     // slices per block
  ShiftTable T;         // truncation of the first GEMM's fixed-point sum, by s
};

__global__ void __launch_bounds__(kSplitXThreads, kSplitXMinBlocks) split_xblocks_kernel(const long long *__restrict__ R, int naux,
                                                                       int nao, int nocc, int nslices, XScale xs,
                                                                       const int *__restrict__ rowE,
                                                                       int *__restrict__ eX,
                                                                       uint16_t *__restrict__ Xd, long long kb_ld,
                                                                       int nblk) {
  extern __shared__ int sh_e[];  // [kBlock] (P, mu) exponents + base, then [nocc] orbital exponents
  const int mu = blockIdx.x;
  const int b = blockIdx.y;
  const int p0 = b * kBlock;
  const int nP = min(kBlock, naux - p0);
  const int klen = nP * nocc;
  const int kpad = (klen + 63) / 64 * 64;
  __shared__ uint64_t red[kSplitXThreads / 32];
  __shared__ int redE[kSplitXThreads / 32];
  __shared__ int e_sh;
  int *eP = sh_e;
  int *eI = sh_e + kBlock;
  {
    const int s1 = xs.s_blk[b];
    const int kbase = -14 - 8 * (s1 - 1) + xs.T.v[s1];
    for (int q = threadIdx.x; q < nP; q += blockDim.x) eP[q] = kbase + xs.eB[(long long)(p0 + q) * nao + mu];
    for (int q = threadIdx.x; q < nocc; q += blockDim.x) eI[q] = xs.eC[q];
  }
  __syncthreads();
  const long long plane = (long long)nblk * nao * kb_ld;
  uint16_t *dst = Xd + ((long long)b * nao + mu) * kb_ld;
  const long long *row0 = R + ((long long)p0 * nao + mu) * nocc;  // element (pl, i) at row0[pl nao nocc + i]
  const long long pstride = (long long)nao * nocc;

  // largest magnitude key (E, M) of the row seen by this thread; E = INT_MIN marks "none yet"
  int bE = INT_MIN;
  uint64_t bM = 0;
  auto take = [&](long long r, int k) {
    if (r == 0) return;
    int E;
    uint64_t M;
    mag_key(r, k, E, M);
    if (E > bE || (E == bE && M > bM)) {
      bE = E;
      bM = M;
    }
  };

  // With the first GEMM's bound g (the largest bitlen(|R|) + k of the row):
  // whether some element reaches 127/128 2^g once rounded to FP64 (only an
  // element with bitlen(|R|) + k == g can: its normalised mantissa M must
  // round to at least 127 2^46 on 53 bits, i.e. M >= 127 2^57 - 2^10, the tie
  // going to the even 127 2^46), and whether the bound holds (no element above
  // g, some element at g).  Bits: 1 reaches, 2 above g, 4 at g.
  constexpr uint64_t kTopM = 0xFDFFFFFFFFFFFC00ull;
  int tbits = 0;
  auto thr = [&](long long r, int k, int g) {
    if (r == 0) return;
    const uint64_t u = r < 0 ? (uint64_t)(-(r + 1)) + 1ull : (uint64_t)r;
    const int lz = __clzll((long long)u);
    const int E = 64 - lz + k;
    tbits |= (E > g ? 2 : 0) | (E == g ? (4 | ((u << lz) >= kTopM ? 1 : 0)) : 0);
  };

  // The digits of the whole row (zero digits in the padding) with exponent e;
  // mode 1 takes the magnitude keys of the row's elements on the way, mode 2
  // the threshold bits against the bound g (= e).
  auto digits_pass = [&](int e, auto mode_c) {
    constexpr int mode = decltype(mode_c)::value;
    constexpr bool keys = mode == 1, tb = mode == 2;
    if ((nocc & 1) == 0) {
      const int hp = nocc >> 1;
      constexpr long long kBias = 0x0080808080808080ll;  // 128 in each of the seven low bytes
      constexpr int kU = 2;                                // pairs per thread per iteration (4 measured slower)
      for (int q0 = threadIdx.x; 2 * q0 < kpad; q0 += kU * blockDim.x) {
        longlong2 v[kU];
        int kq[kU];
#pragma unroll
        for (int r = 0; r < kU; ++r) {
          const int q = q0 + r * blockDim.x;
          const int k = 2 * q;
          v[r] = make_longlong2(0, 0);  // N = 0 (padding) gives zero digits
          kq[r] = -1;
          if (k < klen) {
            const int pl = q / hp;
            const int i = k - pl * nocc;
            v[r] = *reinterpret_cast<const longlong2 *>(row0 + pl * pstride + i);
            kq[r] = pl;
          }
        }
#pragma unroll
        for (int r = 0; r < kU; ++r) {
          const int q = q0 + r * blockDim.x;
          const int k = 2 * q;
          if (k >= kpad) continue;
          long long M0 = kBias, M1 = kBias;
          if (kq[r] >= 0) {
            const int i = k - kq[r] * nocc;
            const int kp = eP[kq[r]];
            if (keys) {
              take(v[r].x, kp + eI[i]);
              take(v[r].y, kp + eI[i + 1]);
            }
            if (tb) {
              thr(v[r].x, kp + eI[i], e);
              thr(v[r].y, kp + eI[i + 1], e);
            }
            M0 += scaled_rne_i64(v[r].x, kp + eI[i], e);
            M1 += scaled_rne_i64(v[r].y, kp + eI[i + 1], e);
          }
#pragma unroll
          for (int t = 0; t < kSMax; ++t)
            if (t < nslices)
              *reinterpret_cast<uint32_t *>(dst + (long long)t * plane + k) =
                  bf16x2_of(digit_f32(M0, t), digit_f32(M1, t));
        }
      }
    } else {
      for (int k = threadIdx.x; k < kpad; k += blockDim.x) {
        int d[kSMax];
        if (k < klen) {
          const int pl = k / nocc;
          const int i = k - pl * nocc;
          const long long r = row0[pl * pstride + i];
          if (keys) take(r, eP[pl] + eI[i]);
          if (tb) thr(r, eP[pl] + eI[i], e);
          balanced_digits(scaled_rne_i64(r, eP[pl] + eI[i], e), d);
        } else {
#pragma unroll
          for (int t = 0; t < kSMax; ++t) d[t] = 0;
        }
#pragma unroll
        for (int t = 0; t < kSMax; ++t)
          if (t < nslices) dst[(long long)t * plane + k] = int_to_bf16_bits(d[t]);
      }
    }
  };

  // The row's exponent from the keys of all threads: e_sh (every thread reads it after the barrier).
  auto reduce_keys = [&]() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int E2 = __shfl_xor_sync(0xffffffffu, bE, o);
      const uint64_t M2 = __shfl_xor_sync(0xffffffffu, bM, o);
      if (E2 > bE || (E2 == bE && M2 > bM)) {
        bE = E2;
        bM = M2;
      }
    }
    if ((threadIdx.x & 31) == 0) {
      redE[threadIdx.x >> 5] = bE;
      red[threadIdx.x >> 5] = bM;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (redE[w] > bE || (redE[w] == bE && red[w] > bM)) {
          bE = redE[w];
          bM = red[w];
        }
      // the row's largest |X| is the rounding of its largest exact magnitude
      const uint64_t top = bE == INT_MIN ? 0ull : abs_bits(ldexp_i64((long long)(bM >> 1), bE - 63));
      e_sh = exponent_from_max_bits_dev(top);
      eX[b * nao + mu] = e_sh;
    }
    __syncthreads();
  };

  const int g = rowE ? __ldg(rowE + b * nao + mu) : kRowBoundNone;
  if (rowE && g != kRowBoundNone && g > -1000 && g < 1000) {
    // One read of R: the row's largest |X| lies in [2^(g-1), 2^g] for the first
    // GEMM's bound g, so its exponent is g, or g + 1 when some element reaches
    // 127/128 2^g: digits with g and the threshold bits on the way, a second
    // pass only for a row that reaches it (far from the FP64 range's ends, so
    // that no element near 2^g is flushed).  Should the bound not hold, the
    // exact keys decide, as below.
    digits_pass(g, Mode<2>{});
    __shared__ int tsh;
    if (threadIdx.x == 0) tsh = 0;
    __syncthreads();
    const int wb = __reduce_or_sync(0xffffffffu, tbits);
    if ((threadIdx.x & 31) == 0 && wb) atomicOr(&tsh, wb);
    __syncthreads();
    const int bits = tsh;
    if ((bits & 6) == 4) {
      const int e = (bits & 1) ? g + 1 : g;
      if (threadIdx.x == 0) eX[b * nao + mu] = e;
      if (e != g) digits_pass(e, Mode<0>{});
    } else {
      digits_pass(g, Mode<1>{});
      reduce_keys();
      if (e_sh != g) digits_pass(e_sh, Mode<0>{});
    }
  } else if (rowE) {
    // an all-zero row (or a bound near the FP64 range's ends): the exact keys
    // on the way, a second pass if the exponent differs from the guess
    const int e0 = g == kRowBoundNone ? exponent_from_max_bits_dev(0ull) : g;
    digits_pass(e0, Mode<1>{});
    reduce_keys();
    if (e_sh != e0) digits_pass(e_sh, Mode<0>{});
  } else {
    // two passes: the keys (four loads in flight per thread), then the digits
    if ((nocc & 1) == 0) {
      const int hp = nocc >> 1;
      const int total = nP * hp;
      for (int q0 = threadIdx.x; q0 < total; q0 += kP1 * blockDim.x) {
        longlong2 v[kP1];
        int kp[kP1], ki[kP1];
#pragma unroll
        for (int r = 0; r < kP1; ++r) {
          const int q = q0 + r * blockDim.x;
          if (q < total) {
            const int pl = q / hp;
            const int i = 2 * (q - pl * hp);
            v[r] = *reinterpret_cast<const longlong2 *>(row0 + pl * pstride + i);
            kp[r] = eP[pl];
            ki[r] = i;
          } else {
            v[r] = make_longlong2(0, 0);
            kp[r] = 0;
            ki[r] = 0;
          }
        }
#pragma unroll
        for (int r = 0; r < kP1; ++r) {
          take(v[r].x, kp[r] + eI[ki[r]]);
          take(v[r].y, kp[r] + eI[ki[r] + 1]);
        }
      }
    } else {
      for (int k = threadIdx.x; k < klen; k += blockDim.x) {
        const int pl = k / nocc;
        const int i = k - pl * nocc;
        take(row0[pl * pstride + i], eP[pl] + eI[i]);
      }
    }
    reduce_keys();
    digits_pass(e_sh, Mode<0>{});
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
  const int g = group > 0 ? group : 1;
  if (cols >= kWideRow) {
    split_rows_bf16_kernel<256><<<(unsigned)rows, 256, 0, st>>>(A, rows, cols, ld, nslices, exps, digits, dld,
                                                                 plane_stride, vec2, perm, g);
  } else {
    const int wpb = 8;
    dim3 grid((unsigned)((rows + wpb - 1) / wpb));
    split_rows_bf16_kernel<32><<<grid, 32 * wpb, 0, st>>>(A, rows, cols, ld, nslices, exps, digits, dld,
                                                         plane_stride, vec2, perm, g);
  }
  return cudaGetLastError();
}

cudaError_t launch_split_rows_packed(const double *Bp, int naux, int nao, int nslices, int *exps, uint16_t *digits,
                                     long long dld, long long plane_stride, const int *perm, cudaStream_t st) {
  const long long rows = (long long)naux * nao;
  if (rows <= 0) return cudaSuccess;
  split_rows_packed_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(Bp, rows, nao, nslices, exps, digits, dld,
                                                                        plane_stride, perm);
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

cudaError_t launch_split_xblocks(const long long *R, int naux, int nao, int nocc, int nslices, const int *eB,
                                 const int *eC, const int *s_blk, const ShiftTable &T1, const int *rowE,
                                 int *eX, uint16_t *Xd, long long kb_ld, int nblk, cudaStream_t st) {
  const size_t sm = sizeof(int) * (size_t)(kBlock + nocc);
  static size_t attr = 48 * 1024;
  if (sm > attr) {
    cudaError_t e = cudaFuncSetAttribute(split_xblocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = sm;
  }
  XScale xs{eB, eC, s_blk, T1};
  dim3 grid(nao, nblk);
  split_xblocks_kernel<<<grid, kSplitXThreads, sm, st>>>(R, naux, nao, nocc, nslices, xs, rowE, eX, Xd, kb_ld,
                                                         nblk);
  return cudaGetLastError();
}

cudaError_t launch_kpart_reduce(const long long *Rp, const int *eX, const int *s_blk, ShiftTable shiftT, int nao,
                                int nblk, int nsplit, double *K, cudaStream_t st) {
  dim3 grid((nao + 127) / 128, nao);
  kpart_reduce_kernel<<<grid, 128, 0, st>>>(Rp, eX, s_blk, shiftT, nao, nblk, nsplit, K);
  return cudaGetLastError();
}

}  // namespace df
