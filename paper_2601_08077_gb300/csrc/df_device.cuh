// Device helpers shared by the libdf kernels: integer-only FP64 bit
// manipulation (GB300's FP64 pipe is narrow, so the split and the
// recombination epilogues never touch it), and the balanced INT8 digit
// expansion of Section 3.2.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace df {

constexpr int kSMax = 8;            // digits per value
constexpr int kBlock = 128;         // auxiliary functions per block

#ifdef __CUDACC__
// Row exponent from the bit pattern of max|row| (a non-negative double):
// the smallest e with vmax < 127/128 * 2^e; 0 for a zero row.
__device__ inline int exponent_from_max_bits_dev(uint64_t bits) {
  if (bits == 0) return 0;
  int E = (int)((bits >> 52) & 0x7FF);
  uint64_t m = bits & ((1ull << 52) - 1);
  if (E == 0) {
    int lz = __clzll((long long)m) - 11;
    m <<= lz;
    E = 1 - lz;
    m &= ((1ull << 52) - 1);
  }
  m |= (1ull << 52);
  return (E - 1023) + 1 + (m >= (127ull << 46) ? 1 : 0);
}

// N = RNE(v * 2^(63-e)) as int64, for |v| < 127/128 2^e.  Integer-only.
__device__ inline long long scaled_rne(uint64_t bits, int e) {
  int E = (int)((bits >> 52) & 0x7FF);
  uint64_t m = bits & ((1ull << 52) - 1);
  if (E == 0) {
    if (m == 0) return 0;
    E = 1;  // subnormal: value = m 2^(1-1075)
  } else {
    m |= (1ull << 52);
  }
  // |v| 2^(63-e) = m 2^(E - 1075 + 63 - e)
  int sh = E - 1012 - e;
  uint64_t n;
  if (sh >= 0) {
    n = m << sh;  // sh <= 10 by the headroom, so n < 2^63
  } else {
    int k = -sh;
    if (k >= 64) {
      n = 0;
    } else {
      uint64_t q = m >> k;
      uint64_t rem = m & ((1ull << k) - 1);
      uint64_t half = 1ull << (k - 1);
      if (rem > half || (rem == half && (q & 1))) q += 1;
      n = q;
    }
  }
  long long N = (long long)n;
  return (bits >> 63) ? -N : N;
}

// Balanced digits of N: d[7..1] in [-128,127] from the bottom, d[0] the rest.
// Taking them from the bottom, digit k is ((N_k + 128) mod 256) - 128 and
// N_{k+1} = floor((N_k + 128) / 256), so with M = N + 128 (1 + 256 + ... +
// 256^6) every low digit is a plain byte of M minus 128 and the top digit is
// M >> 56 (arithmetic; |N| < 127 2^56 keeps M inside int64).
__device__ inline void balanced_digits(long long N, int d[kSMax]) {
  const long long M = N + 0x0080808080808080ll;
  d[0] = (int)(M >> 56);
#pragma unroll
  for (int t = 1; t < kSMax; ++t) d[t] = (int)((M >> (8 * (kSMax - 1 - t))) & 0xFF) - 128;
}

// Exact bf16 bit pattern of a small integer |d| <= 256 (no rounding needed).
// The float is formed as (1.5 2^23 + d) - 1.5 2^23: an integer add on the bit
// pattern (one ulp is 1 there) and one exact FP32 subtraction, both full-rate,
// instead of an int-to-float conversion.
__device__ inline uint16_t int_to_bf16_bits(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return (uint16_t)(__float_as_uint(f) >> 16);
}

// Magnitude key of R 2^k (R != 0): |R| 2^k = M 2^(E - 64) with M normalised
// (top bit set).  Keys compare lexicographically (E, then M) like the exact
// magnitudes, and rounding to FP64 is monotone, so the largest |fl64(R 2^k)|
// of a row is the rounding of its largest key (ldexp_i64(M >> 1, E - 63):
// M's lowest bit is always zero).
__device__ inline void mag_key(long long R, int k, int &E, uint64_t &M) {
  const uint64_t u = R < 0 ? (uint64_t)(-(R + 1)) + 1ull : (uint64_t)R;
  const int lz = __clzll((long long)u);
  E = 64 - lz + k;
  M = u << lz;
}

// N = RNE(fl64(R 2^k) 2^(63-e)) as int64, where fl64 rounds to nearest even
// on 53 bits and flushes results below the normal range to zero exactly as
// ldexp_i64 does; the same value as scaled_rne(bits of ldexp_i64(R, k), e),
// in one pass of integer operations.  Requires |fl64(R 2^k)| < 127/128 2^e.
__device__ inline long long scaled_rne_i64(long long R, int k, int e) {
  if (R == 0) return 0;
  uint64_t u = R < 0 ? (uint64_t)(-(R + 1)) + 1ull : (uint64_t)R;
  const int nb = 64 - __clzll((long long)u);
  int ex = nb - 1 + k;  // exponent of the leading bit
  int sh1 = 0;
  if (nb > 53) {
    sh1 = nb - 53;
    uint64_t q = u >> sh1;
    const uint64_t rem = u & ((1ull << sh1) - 1);
    const uint64_t half = 1ull << (sh1 - 1);
    if (rem > half || (rem == half && (q & 1))) {
      q += 1;
      if (q == (1ull << 53)) {
        q >>= 1;
        sh1 += 1;
        ex += 1;
      }
    }
    u = q;
  }
  if (ex + 1023 <= 0) return 0;  // below the normal range: fl64 flushes to zero
  const int sh2 = sh1 + k + 63 - e;
  uint64_t n;
  if (sh2 >= 0) {
    n = u << sh2;
  } else {
    const int r = -sh2;
    if (r >= 64) {
      n = 0;
    } else {
      uint64_t q = u >> r;
      const uint64_t rem = u & ((1ull << r) - 1);
      const uint64_t half = 1ull << (r - 1);
      if (rem > half || (rem == half && (q & 1))) q += 1;
      n = q;
    }
  }
  return R < 0 ? -(long long)n : (long long)n;
}

// Correctly rounded fp64 of R * 2^k (R int64) by integer operations only.
// Results below the normal range are flushed to signed zero (never met:
// the scales of the DF tensors stay far from 2^-1022).
__device__ inline double ldexp_i64(long long R, int k) {
  if (R == 0) return 0.0;
  uint64_t sign = R < 0 ? (1ull << 63) : 0ull;
  uint64_t u = R < 0 ? (uint64_t)(-(R + 1)) + 1ull : (uint64_t)R;
  int nbits = 64 - __clzll((long long)u);
  uint64_t mant;
  int exp2 = nbits - 1 + k;  // value = 1.xxx * 2^exp2
  if (nbits <= 53) {
    mant = u << (53 - nbits);
  } else {
    int sh = nbits - 53;
    mant = u >> sh;
    uint64_t rem = u & ((1ull << sh) - 1);
    uint64_t half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1))) {
      mant += 1;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        exp2 += 1;
      }
    }
  }
  int be = exp2 + 1023;
  if (be <= 0) return __longlong_as_double((long long)sign);
  if (be >= 2047) return __longlong_as_double((long long)(sign | (0x7FFull << 52)));
  uint64_t bits = sign | ((uint64_t)be << 52) | (mant & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

__device__ inline uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
#endif

}  // namespace df
