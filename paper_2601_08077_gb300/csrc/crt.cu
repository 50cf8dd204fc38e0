// CRT variant of the emulated FP64 GEMM: Ozaki scheme II (Ozaki, Uchino and
// Imamura, 2025), the INT8 alternative to slicing that Section 2.3 of the
// paper names, on the same tensor-core slice GEMM.  Section 4.5 of the paper
// notes that such a library takes a count of moduli rather than an accuracy;
// here the operand width q follows exactly from the moduli and K, so a level
// of Table 1 maps to a modulus count (df_crt_moduli_for_bits).
//
//   moduli   m_1 > m_2 > ... : integers <= 256 taken greedily downwards, each
//            coprime to the ones before; M = m_1 ... m_n < 2^128 (n <= 16)
//   width    q = the largest integer <= 63 with K 2^(2q-1) < M
//   operands e = smallest integer with max|row| < 127/128 2^e (0 for a zero
//            row); A' = RNE(A 2^(q-1-e)) per row, |A'| < 2^62
//   residues a_i = A' mod m_i in [-floor((m_i-1)/2), floor(m_i/2)] (BF16-exact)
//   GEMMs    S_i = a_i b_i^T exactly (products <= 2^14, FP32 chunks of 1024),
//            y_i = S_i mod m_i in the slice GEMM's epilogue (one byte each)
//   CRT      P' = the integer in (-M/2, M/2] with P' = y_i (mod m_i) for all i
//   result   fl64(P' 2^(e_r + f_c - 2(q-1))), one rounding to nearest even
//
// The residues come from the balanced base-256 digits of A' (the digits of the
// slice scheme): A' = sum_j b_j 256^j with signed bytes b_j, so A' mod m is
// congruent to two 4-way signed byte dot products (dp4a) with the centred
// weights 256^j mod m, a sum below 2^17 that one Barrett step reduces.  The
// reconstruction accumulates sum_i y_i W_i (W_i the CRT weights) in 32-bit
// limbs, estimates the quotient by M in FP32 and finishes in 128-bit integers.
// No FP64 instruction is used: GB300's FP64 pipe is narrow.
#include "df_internal.h"

#include <cmath>
#include <cstring>

namespace df {

namespace {

struct CrtTab {
  int n;                            // moduli
  int q1;                           // q - 1
  int mod[kCrtMaxModuli];
  uint32_t magic[kCrtMaxModuli];    // ceil(2^32 / m)
  int off17[kCrtMaxModuli];         // a multiple of m >= 2^17
  int wlo[kCrtMaxModuli];           // centred 256^j mod m, j = 0..3, one signed byte each
  int whi[kCrtMaxModuli];           // j = 4..7
  uint32_t W[kCrtMaxModuli][4];     // CRT weights (M/m_i) ((M/m_i)^-1 mod m_i), 32-bit limbs
  uint32_t M[4];                    // product of the moduli, 32-bit limbs
  float f[4];                       // 2^(32k - sc), or 0 where a limb cannot matter
  float invM;                       // 2^sc / M
};

typedef unsigned __int128 u128;

int greedy_moduli(int n, int *out) {
  int k = 0;
  for (int m = 256; m >= 2 && k < n; --m) {
    bool ok = true;
    for (int j = 0; j < k && ok; ++j) {
      int a = m, b = out[j];
      while (b) {
        const int t = a % b;
        a = b;
        b = t;
      }
      ok = a == 1;
    }
    if (ok) out[k++] = m;
  }
  return k;
}

int bitlen128(u128 v) {
  int b = 0;
  while (v) {
    v >>= 1;
    ++b;
  }
  return b;
}

// q for K-term sums with n moduli (0 if the arguments admit none >= 2).
int operand_bits(long long K, int n) {
  if (K < 1 || K > (1ll << 26) || n < 2 || n > kCrtMaxModuli) return 0;
  int mods[kCrtMaxModuli];
  if (greedy_moduli(n, mods) != n) return 0;
  u128 M = 1;
  for (int i = 0; i < n; ++i) M *= (u128)mods[i];
  // K 2^(2q-1) < M  <=>  2^(2q-1) <= floor((M - 1) / K)  <=>  q <= bitlen / 2
  const u128 D = (M - 1) / (u128)K;
  int q = bitlen128(D) / 2;
  if (q > 63) q = 63;
  return q >= 2 ? q : 0;
}

bool make_tab(long long K, int n, CrtTab *t) {
  std::memset(t, 0, sizeof(*t));
  const int q = operand_bits(K, n);
  if (!q) return false;
  t->n = n;
  t->q1 = q - 1;
  greedy_moduli(n, t->mod);
  u128 M = 1;
  for (int i = 0; i < n; ++i) M *= (u128)t->mod[i];
  for (int i = 0; i < n; ++i) {
    const int m = t->mod[i];
    t->magic[i] = (uint32_t)(0xFFFFFFFFu / (uint32_t)m + 1u);
    t->off17[i] = ((1 << 17) + m - 1) / m * m;
    int lo = 0, hi = 0, w = 1 % m;
    for (int j = 0; j < 8; ++j) {
      const int c = w > m / 2 ? w - m : w;  // centred, in [-128, 127]
      if (j < 4)
        lo |= (c & 0xFF) << (8 * j);
      else
        hi |= (c & 0xFF) << (8 * (j - 4));
      w = (w * 256) % m;
    }
    t->wlo[i] = lo;
    t->whi[i] = hi;
    const u128 c = M / (u128)m;
    const int cm = (int)(c % (u128)m);
    int inv = 0;
    for (int x = 1; x < m; ++x)
      if ((cm * x) % m == 1) {
        inv = x;
        break;
      }
    const u128 Wi = c * (u128)inv;  // < M: c inv < (M / m) m
    for (int k = 0; k < 4; ++k) t->W[i][k] = (uint32_t)(Wi >> (32 * k));
  }
  for (int k = 0; k < 4; ++k) t->M[k] = (uint32_t)(M >> (32 * k));
  // scale the FP32 estimate of V = sum y_i W_i < 2^12 M so it stays below 2^100
  const int bl = bitlen128(M);
  const int sc = bl + 12 > 100 ? bl + 12 - 100 : 0;
  for (int k = 0; k < 4; ++k) {
    const int ex = 32 * k - sc;
    t->f[k] = (ex >= -126 && ex <= 127) ? std::ldexp(1.0f, ex) : 0.0f;
  }
  long double Ml = 0.0L;
  for (int k = 3; k >= 0; --k) Ml = Ml * 4294967296.0L + (long double)t->M[k];
  t->invM = (float)(std::ldexp(1.0L, sc) / Ml);
  return true;
}

__device__ __forceinline__ uint64_t abs_bits(double v) {
  return (uint64_t)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Largest absolute bit pattern over the TPR threads of a row (a warp, or the
// whole 256-thread block through shared memory).
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

// RNE(v 2^(q1 - e)) as int64 for |v| < 127/128 2^e and q1 <= 62.  Integer-only.
__device__ __forceinline__ long long scaled_rne_q(uint64_t bits, int e, int q1) {
  int E = (int)((bits >> 52) & 0x7FF);
  uint64_t m = bits & ((1ull << 52) - 1);
  if (E == 0) {
    if (m == 0) return 0;
    E = 1;
  } else {
    m |= (1ull << 52);
  }
  // |v| 2^(q1 - e) = m 2^(E - 1075 + q1 - e)
  const int sh = E - 1075 + q1 - e;
  uint64_t n;
  if (sh >= 0) {
    n = m << sh;  // sh <= q1 - 53 by the headroom
  } else {
    const int k = -sh;
    if (k >= 64) {
      n = 0;
    } else {
      uint64_t q = m >> k;
      const uint64_t rem = m & ((1ull << k) - 1);
      const uint64_t half = 1ull << (k - 1);
      if (rem > half || (rem == half && (q & 1))) q += 1;
      n = q;
    }
  }
  const long long N = (long long)n;
  return (bits >> 63) ? -N : N;
}

// Centred residue of the integer whose balanced digit words are (hi, lo):
// S = sum_j b_j (256^j mod m) has |S| <= 8 128^2 = 2^17; S + off17 >= 0 is
// reduced by a Barrett step (the high word of v ceil(2^32 / m) is floor(v / m)
// or one more).
__device__ __forceinline__ int residue(int lo, int hi, const CrtTab &t, int i) {
  const int S = __dp4a(lo, t.wlo[i], __dp4a(hi, t.whi[i], 0));
  const int m = t.mod[i];
  const uint32_t v = (uint32_t)(S + t.off17[i]);
  int r = (int)(v - __umulhi(v, t.magic[i]) * (uint32_t)m);
  if (r < 0) r += m;
  return r > (m >> 1) ? r - m : r;
}

// TPR threads per row (a warp, or the whole block for wide rows): exponent,
// scaled integers, residue planes.  kInspect writes the residues as int16
// (inspection entry point), else BF16 bits.
template <bool kInspect, int TPR>
__global__ void __launch_bounds__(256)
    crt_split_rows_kernel(const double *__restrict__ A, long long rows, int cols, long long ld, const CrtTab t,
                          int *__restrict__ exps, uint16_t *__restrict__ planes, long long dld, long long pstride) {
  const int lane = threadIdx.x & (TPR - 1);
  const long long r = (long long)blockIdx.x * (blockDim.x / TPR) + (threadIdx.x / TPR);
  if (r >= rows) return;  // uniform over a row's threads
  const double *row = A + r * ld;
  uint64_t mx = 0;
  for (int c = lane; c < cols; c += TPR) {
    const uint64_t a = abs_bits(__ldg(row + c));
    mx = a > mx ? a : mx;
  }
  mx = row_max_u64<TPR>(mx);
  const int e = exponent_from_max_bits_dev(mx);
  if (lane == 0) exps[r] = e;
  uint16_t *drow = planes + r * dld;
  // four columns per lane per step: four independent chains per residue
  for (int c = 4 * lane; c < cols; c += 4 * TPR) {
    const int nv = cols - c < 4 ? cols - c : 4;
    int lo[4], hi[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const uint64_t b = h < nv ? (uint64_t)__double_as_longlong(row[c + h]) : 0ull;
      // balanced digits: byte j of Mg is b_j + 128 for j < 7, the top byte is b_7
      const long long Mg = scaled_rne_q(b, e, t.q1) + 0x0080808080808080ll;
      lo[h] = (int)((uint32_t)Mg ^ 0x80808080u);
      hi[h] = (int)((uint32_t)((unsigned long long)Mg >> 32) ^ 0x00808080u);
    }
    for (int i = 0; i < t.n; ++i) {
      uint32_t v[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int rr = residue(lo[h], hi[h], t, i);
        v[h] = kInspect ? (uint32_t)(uint16_t)(int16_t)rr : (uint32_t)int_to_bf16_bits(rr);
      }
      uint16_t *dst = drow + (long long)i * pstride + c;
      if (nv == 4 && ((reinterpret_cast<uintptr_t>(dst) & 7) == 0)) {
        *reinterpret_cast<uint2 *>(dst) = make_uint2(v[0] | (v[1] << 16), v[2] | (v[3] << 16));
      } else {
        for (int h = 0; h < nv; ++h) dst[h] = (uint16_t)v[h];
      }
    }
  }
}

// P' from the residue bytes of one element, then fl64(P' 2^k).
__device__ __forceinline__ double crt_value(const uint8_t *y, long long plane, const CrtTab &t, int k) {
  uint64_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;  // V = sum_j a_j 2^(32j), each a_j < 2^44
  for (int i = 0; i < t.n; ++i) {
    const uint64_t v = y[i * plane];
    a0 += v * t.W[i][0];
    a1 += v * t.W[i][1];
    a2 += v * t.W[i][2];
    a3 += v * t.W[i][3];
  }
  // V / M < 4096; the FP32 estimate is within 1/64 of it, so floor is off by at most 1
  const float vf = (float)a0 * t.f[0] + (float)a1 * t.f[1] + (float)a2 * t.f[2] + (float)a3 * t.f[3];
  const long long qe = (long long)__float2int_rd(vf * t.invM);
  // R = V - qe M in 128-bit two's complement (it lies in (-M, 2M))
  const u128 R0 = (u128)(long long)((long long)a0 - qe * (long long)t.M[0]) +
                  ((u128)(long long)((long long)a1 - qe * (long long)t.M[1]) << 32) +
                  ((u128)(long long)((long long)a2 - qe * (long long)t.M[2]) << 64) +
                  ((u128)(long long)((long long)a3 - qe * (long long)t.M[3]) << 96);
  __int128 R = (__int128)R0;
  const __int128 M = (__int128)(((u128)t.M[3] << 96) | ((u128)t.M[2] << 64) | ((u128)t.M[1] << 32) | (u128)t.M[0]);
  if (R < 0)
    R += M;
  else if (R >= M)
    R -= M;
  if (2 * R > M) R -= M;  // the representative in (-M/2, M/2]
  if (R == 0) return 0.0;
  const bool neg = R < 0;
  const u128 u = neg ? (u128)(-R) : (u128)R;
  const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
  if (hi == 0 && lo < (1ull << 63)) return ldexp_i64(neg ? -(long long)lo : (long long)lo, k);
  // 63 leading bits plus a sticky bit: rounding them once gives the rounding of u
  const int nb = hi ? 128 - __clzll((long long)hi) : 64;
  const int sh = nb - 63;
  uint64_t win = (uint64_t)(u >> sh);
  if (u & (((u128)1 << sh) - 1)) win |= 1ull;
  return ldexp_i64(neg ? -(long long)win : (long long)win, k + sh);
}

__global__ void __launch_bounds__(256)
    crt_reconstruct_kernel(const uint8_t *__restrict__ Y, int M, int N, long long ldy, long long plane,
                           const int *__restrict__ ea, const int *__restrict__ eb, const CrtTab t,
                           double *__restrict__ out, long long ldo) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int ebn = eb[n];
  for (int m = blockIdx.y; m < M; m += gridDim.y)
    out[(long long)m * ldo + n] = crt_value(Y + (long long)m * ldy + n, plane, t, ea[m] + ebn - 2 * t.q1);
}

cudaError_t launch_crt_split(const double *A, long long rows, int cols, long long ld, const CrtTab &t, int *exps,
                             uint16_t *planes, long long dld, long long pstride, bool inspect, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (cols >= kWideRow) {
    const dim3 grid((unsigned)rows);
    if (inspect)
      crt_split_rows_kernel<true, 256><<<grid, 256, 0, st>>>(A, rows, cols, ld, t, exps, planes, dld, pstride);
    else
      crt_split_rows_kernel<false, 256><<<grid, 256, 0, st>>>(A, rows, cols, ld, t, exps, planes, dld, pstride);
  } else {
    const dim3 grid((unsigned)((rows + 7) / 8));
    if (inspect)
      crt_split_rows_kernel<true, 32><<<grid, 256, 0, st>>>(A, rows, cols, ld, t, exps, planes, dld, pstride);
    else
      crt_split_rows_kernel<false, 32><<<grid, 256, 0, st>>>(A, rows, cols, ld, t, exps, planes, dld, pstride);
  }
  return cudaGetLastError();
}

long long round_up_ll(long long v, long long a) { return (v + a - 1) / a * a; }

// Split both operands, run the per-modulus slice GEMMs (residue bytes in Y,
// [nmod][M][ldy]) and, if out != NULL, reconstruct.  Y_user (optional) gets
// the residues as [nmod][M][N]; ea_user / eb_user the exponents.
df_status crt_gemm(const double *A, const double *B, int M, int N, int K, int nmod, double *out, uint8_t *Y_user,
                   int32_t *ea_user, int32_t *eb_user, cudaStream_t st) {
  if (!A || !B || M <= 0 || N <= 0 || K <= 0) return DF_ERR_ARG;
  CrtTab t;
  if (!make_tab(K, nmod, &t)) return DF_ERR_ARG;
  const long long ld = round_up_ll(K, 8);
  const long long ldy = round_up_ll(N, 16);
  // A B^T with B == A (a Gram matrix such as K_b = X_b X_b^T): one split serves both sides
  const bool same = A == B && M == N;
  uint16_t *Ad = nullptr, *Bd = nullptr;
  uint8_t *Y = nullptr;
  int *ea = nullptr, *eb = nullptr, *status = nullptr;
  df_status rs = DF_OK;
  cudaError_t e = scratch_malloc((void **)&Ad, sizeof(uint16_t) * (size_t)nmod * M * ld, st);
  if (e == cudaSuccess && !same) e = scratch_malloc((void **)&Bd, sizeof(uint16_t) * (size_t)nmod * N * ld, st);
  if (e == cudaSuccess) e = scratch_malloc((void **)&Y, (size_t)nmod * M * ldy, st);
  if (e == cudaSuccess) e = scratch_malloc((void **)&ea, sizeof(int) * M, st);
  if (e == cudaSuccess && !same) e = scratch_malloc((void **)&eb, sizeof(int) * N, st);
  if (e == cudaSuccess) e = scratch_malloc((void **)&status, sizeof(int), st);
  if (e == cudaErrorMemoryAllocation) rs = DF_ERR_OOM;
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = launch_crt_split(A, M, K, K, t, ea, Ad, ld, (long long)M * ld, false, st);
  if (e == cudaSuccess && !same) e = launch_crt_split(B, N, K, K, t, eb, Bd, ld, (long long)N * ld, false, st);
  const uint16_t *Bplanes = same ? Ad : Bd;
  const int *ebx = same ? ea : eb;
  if (e == cudaSuccess) {
    CUtensorMap ta, tb;
    if (!make_tmap_bf16(&ta, Ad, K, M, nmod, ld, (long long)M * ld) ||
        !make_tmap_bf16(&tb, Bplanes, K, N, nmod, ld, (long long)N * ld)) {
      rs = DF_ERR_CUDA;
    } else {
      SgParams p;
      std::memset(&p, 0, sizeof(p));
      p.layout = kLayoutCrt;
      p.mode = kModeMod;
      p.nt_m = (M + kTile - 1) / kTile;
      p.nt_n = (N + kTile - 1) / kTile;
      p.nunits = nmod * p.nt_m * p.nt_n;
      p.m_valid = M;
      p.n_valid = N;
      p.ktiles = (K + kKTile - 1) / kKTile;
      p.s_fixed = 1;
      p.shiftT[1] = fixed_point_shift(1, (long long)p.ktiles * kKTile);  // 0: the sums are exact
      p.out = reinterpret_cast<double *>(Y);
      p.out_ld = ldy;
      p.out_blk = (long long)M * ldy;
      p.status = status;
      for (int i = 0; i < nmod; ++i) p.crt_mod[i] = t.mod[i];
      if (p.shiftT[1] != 0 || (long long)p.nunits > (1ll << 30)) rs = DF_ERR_ARG;
      else e = launch_slice_gemm(p, ta, tb, st);
    }
  }
  if (e == cudaSuccess && rs == DF_OK && out) {
    const dim3 grid((unsigned)((N + 255) / 256), (unsigned)(M < 65535 ? M : 65535));
    crt_reconstruct_kernel<<<grid, 256, 0, st>>>(Y, M, N, ldy, (long long)M * ldy, ea, ebx, t, out, N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && rs == DF_OK && Y_user)
    e = cudaMemcpy2DAsync(Y_user, N, Y, ldy, N, (size_t)nmod * M, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && rs == DF_OK && ea_user)
    e = cudaMemcpyAsync(ea_user, ea, sizeof(int) * M, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && rs == DF_OK && eb_user)
    e = cudaMemcpyAsync(eb_user, ebx, sizeof(int) * N, cudaMemcpyDeviceToDevice, st);
  int h = 0;
  if (e == cudaSuccess && rs == DF_OK) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  for (void *ptr : {(void *)Ad, (void *)Bd, (void *)Y, (void *)ea, (void *)eb, (void *)status})
    if (ptr) cudaFreeAsync(ptr, st);
  const cudaError_t es = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = es;
  if (rs != DF_OK) return rs;
  if (e != cudaSuccess) return DF_ERR_CUDA;
  return h ? DF_ERR_TIMEOUT : DF_OK;
}

}  // namespace

}  // namespace df

extern "C" {

int df_crt_modulus(int i) {
  int mods[df::kCrtMaxModuli];
  if (i < 0 || i >= df::kCrtMaxModuli) return 0;
  df::greedy_moduli(df::kCrtMaxModuli, mods);
  return mods[i];
}

int df_crt_operand_bits(long long K, int nmod) { return df::operand_bits(K, nmod); }

int df_crt_moduli_for_bits(long long K, int bits) {
  for (int n = 2; n <= df::kCrtMaxModuli; ++n)
    if (df::operand_bits(K, n) >= bits + 1) return n;
  return 0;
}

df_status df_crt_split_rows(const double *A, int rows, int cols, int ld, int nmod, int32_t *exps, int16_t *res,
                            void *stream) {
  if (!A || !exps || !res || rows < 0 || cols <= 0 || ld < cols) return DF_ERR_ARG;
  df::CrtTab t;
  if (!df::make_tab(cols, nmod, &t)) return DF_ERR_ARG;
  const cudaError_t e = df::launch_crt_split(A, rows, cols, ld, t, exps, reinterpret_cast<uint16_t *>(res), cols,
                                             (long long)rows * cols, true, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DF_OK : DF_ERR_CUDA;
}

df_status df_crt_residue_products(const double *A, const double *B, int M, int N, int K, int nmod, uint8_t *Y,
                                  int32_t *ea, int32_t *eb, void *stream) {
  if (!Y) return DF_ERR_ARG;
  return df::crt_gemm(A, B, M, N, K, nmod, nullptr, Y, ea, eb, reinterpret_cast<cudaStream_t>(stream));
}

df_status df_emulated_gemm_crt(const double *A, const double *B, int M, int N, int K, int nmod, double *out,
                               void *stream) {
  if (!out) return DF_ERR_ARG;
  return df::crt_gemm(A, B, M, N, K, nmod, out, nullptr, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
