// Slice GEMM on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// Computes, for an output tile of 128 (A-side rows) x 128 (B-side rows), the
// exact slice-pair sums of Section 3.2
//
//     S_g = sum_{t+u=g} A_t B_u^T,   g = 0 .. s-1,
//
// where A_t, B_u are INT8 digit planes (row-major, K contiguous), and folds
// them into the fixed-point value R = sum_g 2^(8(s-1-g)) S_g, which the
// epilogue turns into FP64 with the per-row / per-column power-of-two scales.
//
// GB300 mapping.  ptxas rejects tcgen05 .kind::i8 on sm_103a, so the digits
// are stored as BF16 (every integer in [-256, 256] is exact in BF16) and run
// through tcgen05.mma .kind::f16 with FP32 accumulators in TMEM.  A product of
// two digits is at most 2^14 in magnitude, so an accumulation of at most 1024
// products stays within 2^24 and is exact in FP32; the MMA warp therefore
// closes an accumulator "chunk" every <= 1024 products (<= 16 pipeline
// stages) and the epilogue warps add it, converted to integers and shifted by
// its group's weight, into an int64 fixed-point total held in registers (64
// per thread).  One tcgen05.mma (M = 128, N = 256) computes two slice pairs
// (t, u) and (t, u+1) at once: its B operand is B_u stacked on B_{u+1}, so
// TMEM columns 0-255 hold one accumulator buffer of 2 x 128 columns and
// columns 256-511 the second (the tensor core fills one while the epilogue
// drains the other).
//
// Warp roles (384 threads, one CTA per SM, persistent over work units):
//   warp 0      TMA producer: 128x64 BF16 boxes of A_t, B_u and B_{u+1},
//               128B swizzle, into a 4-stage ring (48 KB per stage) guarded
//               by mbarriers;
//   warp 1      TMEM allocation and the single-thread tcgen05.mma issuer;
//   warps 2, 3  idle (they give their registers to the epilogue: setmaxnreg);
//   warps 4..11 epilogue; warp w reads TMEM lanes 32*(w%4)..+31 (tile rows)
//               and columns 64*((w-4)/4)..+63 of each 128-column half.
//
// CTA-pair mode (cluster of two): rank 0's MMA issuer runs tcgen05.mma
// .cta_group::2 with M = 256 over two output tiles that share the B operand;
// each CTA stages its own A tile and one of the two stacked B tiles (a
// 6-stage ring of 32 KB), both CTAs' copies complete on rank 0's barriers,
// the commits arrive on both CTAs' barriers, and each CTA drains its own TMEM.
//
// Every mbarrier wait is bounded (4 s of wall clock); a wait that runs out
// sets a shared abort flag and bit 1 of the device status word, every role
// leaves its loop, the producer waits (bounded) for its copies in flight, the
// MMA issuer waits (bounded) for its MMAs, and the TMEM is freed.
#include "df_internal.h"

#include <cstdio>
#include <cstring>

namespace df {

namespace {

constexpr int kStages = 4;
constexpr int kTileBytes = kTile * kKTile * 2;        // one 128 x 64 BF16 box, 16 KB
constexpr int kStageBytes = 3 * kTileBytes;           // A_t tile + two stacked B tiles
// CTA-pair mode (cta_group::2): a CTA stages its own A_t tile and one of the
// two stacked B tiles, so a stage is 32 KB and six fit in the space of the
// four 48 KB stages (seven measured no faster on GB300).
constexpr int kStagesP = 6;
constexpr int kStageBytesP = 2 * kTileBytes;
constexpr int kThreads = 384;                         // 12 warps
constexpr int kEpiWarp0 = 4;
constexpr int kEpiWarps = 8;
constexpr int kAccBufs = 2;
constexpr uint32_t kAccCols = 256;                    // one accumulator buffer: two 128-column halves
constexpr uint32_t kTmemCols = 512;
constexpr int kChunkStages = kMaxChunk / kKTile;      // 16 stages = 1024 products
constexpr uint64_t kTimeoutNs = 4000000000ull;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*barriers*/ + 1024 /*alignment slack*/;
constexpr int kSmemBytesP = kStagesP * kStageBytesP + 1024 /*barriers*/ + 1024 /*alignment slack*/;
static_assert(kSmemBytesP <= 232448, "pair ring must fit the 227 KB opt-in shared memory of a CTA");
// CRT variant (kModeMod): one B tile per stage and short units (one plane,
// K / 64 stages each) streaming a large A operand, so the ring is deepened
// to keep more DRAM reads in flight.
constexpr int kStagesM = 7;
constexpr int kSmemBytesM = kStagesM * kStageBytesP + 1024 /*barriers*/ + 1024 /*alignment slack*/;
static_assert(kSmemBytesM <= 232448, "CRT ring must fit the 227 KB opt-in shared memory of a CTA");
// Register split (setmaxnreg): warps 0-3 drop to 56, the 8 epilogue warps rise
// to 224; 128*56 + 256*224 = 64512 = 384 threads * 168 registers at launch.
constexpr int kRegsLow = 56;
constexpr int kRegsHigh = 224;
static_assert(128 * kRegsLow + 256 * kRegsHigh <= kThreads * 168, "register split exceeds the launch's registers");

// BF16 x BF16 -> FP32, both operands K-major, M = 128, N = 128 or 256
// (instruction descriptor of tcgen05.mma .kind::f16: D fmt bits 4-5, A fmt
// 7-9, B fmt 10-12, N>>3 at 17-22, M>>4 at 24-28).
constexpr uint32_t idesc_for(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}
constexpr uint32_t kIdesc128 = idesc_for(128);
constexpr uint32_t kIdesc256 = idesc_for(256);
// M = 256 across the CTA pair (128 rows of A in each CTA), N = 256 (B rows
// 0-127 from the first CTA's shared memory, 128-255 from the second's).
constexpr uint32_t kIdescPair = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
                                ((uint32_t)(256 >> 4) << 24);

struct Unit {
  int m0, n0, az0, azs, bz0, bzs, kt0, ktiles, s, blk, part;
  // block-sparse K (first exchange GEMM on a screened B): the unit's nonzero
  // K tiles as a bit mask; ktiles then counts its set bits
  int sparse;
  uint32_t kmask;
};

// Index of the unit's i-th K tile: the i-th set bit of the mask when the
// unit is block-sparse, else kt0 + i.
__device__ __forceinline__ int ktile_of(const Unit &w, int i) {
  return w.sparse ? (int)__fns(w.kmask, 0u, i + 1) : w.kt0 + i;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Acquire at cluster scope: the barrier may complete through arrivals or
// copies issued by the other CTA of a pair.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait.  Returns false if the CTA is aborting or the wait ran out.
template <bool kCluster = false>
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                             int *status, bool honour_abort = true,
                                             uint64_t limit_ns = kTimeoutNs) {
  auto poll = [&]() { return kCluster ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity); };
  if (poll()) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (poll()) return true;
    if (honour_abort && *abort_flag) return false;
    if (globaltimer_ns() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicOr(status, 1);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row core
// groups 1024 bytes apart (SBO), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// --- CTA pair (cta_group::2) ---------------------------------------------
// TMA load into this CTA's shared memory that completes its bytes on the
// mbarrier at shared::cluster address `mbar` (rank 0's, for both CTAs).
__device__ __forceinline__ void tma_load_3d_pair(void *dst, const CUtensorMap *map, uint32_t mbar, int c0, int c1,
                                                 int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
      : "memory");
}

// One thread of the first CTA issues the M = 256 MMA for both CTAs.
__device__ __forceinline__ void umma_bf16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive (once the pair's MMAs issued so far are done) on the barrier at the
// same offset in both CTAs of the pair.
__device__ __forceinline__ void umma_commit_pair(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}

// Shared::cluster address of this CTA's variable `p` in CTA `rank`.
__device__ __forceinline__ uint32_t peer_addr(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

// Arrive on a barrier of either CTA of the pair.  Default semantics: what the
// arrival publishes (TMEM reads done) is ordered by the tcgen05 fences around
// it, so no cluster-scope release (a full memory barrier) is needed.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of both CTAs of the cluster.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Tile (i, j) of block-and-split index bs of the second exchange GEMM.
__device__ __forceinline__ Unit kpart_unit(const SgParams &p, int i, int j, int bs) {
  Unit w;
  const int b = bs / p.nsplit;
  const int sp = bs - b * p.nsplit;
  w.m0 = i * kTile;
  w.n0 = j * kTile;
  w.az0 = b;
  w.azs = p.nblk;
  w.bz0 = b;
  w.bzs = p.nblk;
  const int nP = min(kBlock, p.naux - b * kBlock);
  const int kt_b = (nP * p.nocc + kKTile - 1) / kKTile;
  w.kt0 = (int)((long long)kt_b * sp / p.nsplit);
  w.ktiles = (int)((long long)kt_b * (sp + 1) / p.nsplit) - w.kt0;
  w.s = p.s_blk[b];
  w.blk = b;
  w.part = bs;
  w.sparse = 0;
  w.kmask = 0u;
  return w;
}

// Tile (mt, nt) of the grid layouts (kLayoutGrid, kLayoutX, kLayoutXs).
__device__ __forceinline__ Unit grid_unit(const SgParams &p, int mt, int nt) {
  Unit w;
  w.m0 = mt * kTile;
  w.n0 = nt * kTile;
  w.az0 = 0;
  w.azs = 1;
  w.bz0 = 0;
  w.bzs = 1;
  w.kt0 = 0;
  w.part = 0;
  w.ktiles = p.ktiles;
  w.sparse = 0;
  w.kmask = 0u;
  if (p.kmask && (p.layout == kLayoutX || p.layout == kLayoutXs)) {
    // the (P, mu) row tile of B's digits: the n tile (kLayoutX) or the m tile (kLayoutXs)
    const int t = p.layout == kLayoutX ? nt : mt;
    const int ntile = p.layout == kLayoutX ? p.nt_n : p.nt_m;
    w.sparse = 1;
    w.kmask = t < ntile ? p.kmask[t] : 0u;
    w.ktiles = __popc(w.kmask);
  }
  if (p.layout == kLayoutX || p.layout == kLayoutXs) {
    // the (P, mu) rows of a 128-function block: a tile never straddles two blocks
    const long long r0 = p.layout == kLayoutX ? (long long)w.n0 : (long long)w.m0;
    w.blk = (int)(r0 / ((long long)kBlock * p.nao));
    if (w.blk >= p.nblk) w.blk = p.nblk - 1;  // a tile past the last row (pairs): any valid count
    w.s = p.s_blk[w.blk];
  } else {
    w.blk = 0;
    w.s = p.s_fixed;
  }
  return w;
}

__device__ __forceinline__ Unit decode_unit(const SgParams &p, int u) {
  Unit w;
  if (p.layout == kLayoutCrt) {
    // plane-major, so the B tile of a plane is reused from L2 by its m tiles
    const int per = p.nt_m * p.nt_n;
    const int plane = u / per, r = u % per;
    w = grid_unit(p, r % p.nt_m, r / p.nt_m);
    w.az0 = plane;
    w.bz0 = plane;
    w.blk = plane;
    return w;
  }
  if (p.layout == kLayoutKPart) {
    // u -> (block b, K split sp, upper tile pair); block-major for L2 reuse
    const int npairs = p.nt_m * (p.nt_m + 1) / 2;
    const int pr = u % npairs;
    int i = 0, rem = pr;
    while (rem >= p.nt_m - i) {
      rem -= p.nt_m - i;
      ++i;
    }
    return kpart_unit(p, i, i + rem, u / npairs);
  }
  return grid_unit(p, u % p.nt_m, u / p.nt_m);
}

// Tile of CTA `r` (0 or 1) of tile pair `pu` in CTA-pair mode: both tiles
// share the n tile (the B-side operand), their m tiles are 2a and 2a+1.  In
// the second exchange GEMM the pairs of (block, split) bs are (2a + r, j) for
// j = 2a .. nt-1: the pair at j = 2a also computes the lower tile (2a+1, 2a),
// whose values are the transpose of an upper tile and are never read, and an
// m tile past the last one reads zeros and stores nothing.
__device__ __forceinline__ Unit decode_pair(const SgParams &p, int pu, int r) {
  if (p.layout == kLayoutKPart) {
    const int nt = p.nt_m;
    const int na = (nt + 1) / 2;
    const int per = na * (nt - na + 1);  // sum over a < na of (nt - 2a)
    const int pr = pu % per;
    int a = 0, rem = pr;
    while (rem >= nt - 2 * a) {
      rem -= nt - 2 * a;
      ++a;
    }
    return kpart_unit(p, 2 * a + r, 2 * a + rem, pu / per);
  }
  if (p.layout == kLayoutXs) {
    // (P, mu) tiles 2a, 2a+1 (the second may lie past the last: zeros, no
    // stores); the orbital tiles of one pair of (P, mu) tiles run back to
    // back, so its B-digit tiles are reused from L2.  Block-sparse: both CTAs
    // run the union of the two tiles' K tiles (one MMA covers both).
    Unit w = grid_unit(p, 2 * (pu / p.nt_n) + r, pu % p.nt_n);
    if (w.sparse) {
      const int other = 2 * (pu / p.nt_n) + (1 - r);
      if (other < p.nt_m) w.kmask |= p.kmask[other];
      w.ktiles = __popc(w.kmask);
    }
    return w;
  }
  const int h = p.nt_m >> 1;
  return grid_unit(p, 2 * (pu % h) + r, pu / h);
}

// Epilogue store of the 64 output columns n0c..n0c+63 of row m.
// First exchange GEMM: the exact int64 sums of X tile columns n0c..n0c+63
// (rows n = (P, mu)) of orbital m; the X split applies the scales and the
// rounding to FP64.
__device__ __forceinline__ void store64_x(const SgParams &p, int m, int n0c, const long long (&R)[64]) {
  if (m >= p.m_valid) return;
  long long *out = reinterpret_cast<long long *>(p.out);
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    const int n = n0c + j;
    if (n >= p.n_valid) continue;
    out[(long long)n * p.out_ld + m] = R[j];
  }
}

// v mod m for 0 <= v < 2^32 and 2 <= m <= 256 with magic = ceil(2^32 / m):
// the high word of v * magic is floor(v / m) or one more, so one correction.
__device__ __forceinline__ int umod_barrett(uint32_t v, int m, uint32_t magic) {
  const int r = (int)(v - __umulhi(v, magic) * (uint32_t)m);
  return r < 0 ? r + m : r;
}

// R mod m in [0, m) for |R| < 2^40: R = a 2^24 + b with |a| < 2^16 and
// 0 <= b < 2^24; a 2^24 = a c24 (mod m) with c24 = 2^24 mod m, |a c24| < 2^24,
// made non-negative by off24, a multiple of m >= 2^24.
__device__ __forceinline__ int mod_i40(long long R, int m, uint32_t magic, int c24, int off24) {
  const int a = (int)(R >> 24);
  const uint32_t b = (uint32_t)(R & 0xFFFFFF);
  const int r = umod_barrett((uint32_t)(a * c24 + off24), m, magic) + umod_barrett(b, m, magic);
  return r >= m ? r - m : r;
}

// First exchange GEMM: this unit's part of the per-(block, mu) bound on the
// exponent of each X row (SgParams::rowE).  An element's exact sum R with
// exponent sum k has |R 2^k| < 2^E, E = bitlen(|R|) + k, two integer
// operations with no rounding; the row bound is the largest E of its nonzero
// elements.  kModeX: a thread's 64 columns are 64 (P, mu) rows of X and the
// lanes of its warp are orbitals, so each column is maxed over the warp with
// one redux and one lane adds it atomically; kModeXs: the thread's row is one
// (P, mu), its columns orbitals, so it maxes its own values.  Lanes that gave
// up on a wait are not here; the reduction takes the lanes that are.
__device__ __forceinline__ int bit_length(long long r) {
  const uint64_t u = r < 0 ? (uint64_t)(-(r + 1)) + 1ull : (uint64_t)r;
  return 64 - __clzll((long long)u);
}

template <int kMode>
__device__ __forceinline__ void record_row_bound(const SgParams &p, int m, int n0c, const long long (&R)[64],
                                                 int kexp_base, int lane) {
  if constexpr (kMode == kModeX) {
    // v[j]: this lane's bound for column j without the column's exponent
    // eb[n] (the same on every lane, added by the lane that ends up owning the
    // column).  A butterfly reduce-scatter over the warp: at each of five steps
    // a lane keeps half of its columns, sends the other half to its partner
    // and maxes what it receives; the shuffles of a step are independent, and
    // lane L ends with columns 2L and 2L + 1.
    const unsigned active = __activemask();
    const bool mv = m < p.m_valid;
    const int km = kexp_base + (mv ? p.ea[m] : 0);
    int v[64];
#pragma unroll
    for (int j = 0; j < 64; ++j)
      v[j] = (mv && n0c + j < p.n_valid && R[j] != 0) ? bit_length(R[j]) + km : kRowBoundNone;
#pragma unroll
    for (int w = 32; w >= 2; w >>= 1) {
      // w columns held; keep w / 2: the upper half when this lane's bit is set
      const int bit = (w == 32 ? 16 : w == 16 ? 8 : w == 8 ? 4 : w == 4 ? 2 : 1);
      const bool upper = (lane & bit) != 0;
#pragma unroll
      for (int i = 0; i < w; ++i) {
        const int send = upper ? v[i] : v[i + w];
        const int keep = upper ? v[i + w] : v[i];
        const int got = __shfl_xor_sync(active, send, bit);
        v[i] = keep > got ? keep : got;
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = n0c + 2 * lane + h;
      if (v[h] != kRowBoundNone && n < p.n_valid) {
        const int P = n / p.nao, mu = n - P * p.nao;
        atomicMax(p.rowE + (P / kBlock) * p.nao + mu, v[h] + __ldg(p.eb + n));
      }
    }
  } else if constexpr (kMode == kModeXs) {
    if (m >= p.m_valid) return;
    const int km = kexp_base + p.ea[m];
    int best = kRowBoundNone;
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      const int n = n0c + j;
      if (n < p.n_valid && R[j] != 0) best = max(best, bit_length(R[j]) + km + __ldg(p.eb + n));
    }
    if (best != kRowBoundNone) {
      const int P = m / p.nao, mu = m - P * p.nao;
      atomicMax(p.rowE + (P / kBlock) * p.nao + mu, best);
    }
  }
}

template <int kMode>
__device__ __forceinline__ void store64(const SgParams &p, const Unit &w, int m, int n0c, const long long (&R)[64],
                                        int kexp_base, int ea_m) {
  if (kMode == kModeMod) {
    // CRT variant: y = S mod m_plane, one byte per element, row-major per plane
    if (m >= p.m_valid) return;
    const int md = p.crt_mod[w.blk];
    const uint32_t magic = 0xFFFFFFFFu / (uint32_t)md + 1u;
    const int c24 = (int)((1u << 24) % (unsigned)md);
    const int off24 = (int)(((1u << 24) + (unsigned)md - 1u) / (unsigned)md * (unsigned)md);
    uint8_t *out = reinterpret_cast<uint8_t *>(p.out) + (long long)w.blk * p.out_blk + (long long)m * p.out_ld + n0c;
    if (n0c + 64 <= p.n_valid) {
#pragma unroll
      for (int j8 = 0; j8 < 8; ++j8) {
        uint64_t word = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) word |= (uint64_t)mod_i40(R[8 * j8 + j], md, magic, c24, off24) << (8 * j);
        reinterpret_cast<uint64_t *>(out)[j8] = word;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 64; ++j)
        if (n0c + j < p.n_valid) out[j] = (uint8_t)mod_i40(R[j], md, magic, c24, off24);
    }
    return;
  }
  if (kMode == kModeX) {
    store64_x(p, m, n0c, R);
    return;
  }
  if (kMode == kModeXs) {
    // swapped first GEMM: row m = (P, mu), columns n = orbitals, the same X[(P, mu)][i]
    if (m >= p.m_valid) return;
    long long *out = reinterpret_cast<long long *>(p.out) + (long long)m * p.out_ld;
#pragma unroll
    for (int j = 0; j < 64; ++j)
      if (n0c + j < p.n_valid) out[n0c + j] = R[j];
    return;
  }
  if (m >= p.m_valid) return;
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    const int n = n0c + j;
    if (n >= p.n_valid) continue;
    if (kMode == kModeX) {
      p.out[(long long)n * p.out_ld + m] = ldexp_i64(R[j], kexp_base + ea_m + p.eb[n]);
    } else if (kMode == kModeKPart) {
      p.raw[(long long)w.part * p.out_blk + (long long)n * p.out_ld + m] = R[j];
    } else if (kMode == kModeGemm) {
      p.out[(long long)m * p.out_ld + n] = ldexp_i64(R[j], kexp_base + ea_m + p.eb[n]);
    }
  }
}

// K tiles of a unit are taken in ceil(ktiles / 16) chunks of near-equal
// length (at most 16 stages = 1024 products each, the exact FP32 range).
__device__ __forceinline__ int num_chunks(int ktiles) { return (ktiles + kChunkStages - 1) / kChunkStages; }
__device__ __forceinline__ int chunk_begin(int ktiles, int nch, int c) { return ktiles * c / nch; }

// acc + v 2^sh for 0 <= sh <= 30: one widening multiply-add (2^sh fits a
// signed 32-bit multiplier), exact in int64
__device__ __forceinline__ long long mad_pow2(int v, int pow2, long long acc) {
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(v), "r"(pow2), "l"(acc));
  return d;
}

// acc + v 2^sh for 32 <= sh <= 63, modulo 2^64: only the high word changes
__device__ __forceinline__ long long add_high(int v, int sh_hi, long long acc) {
  return (long long)((unsigned long long)acc + ((unsigned long long)((uint32_t)v << sh_hi) << 32));
}

__device__ __forceinline__ long long weigh(int v, int sh) {
  const long long x = (long long)v;
  return sh >= 0 ? (x << sh) : ((x + (1ll << (-sh - 1))) >> (-sh));
}

// The work of one unit is a sequence of "slots": for t = 0..s-1, u0 = 0, 2, 4, ...
// <= s-1-t, the slot computes the slice pairs (t, u0) and, if u0+1 <= s-1-t,
// (t, u0+1) with one N = 256 MMA per K step (B operand = B_u0 stacked on
// B_u0+1); a single pair uses N = 128.  The K tiles of the unit are cut into
// chunks of at most 16 stages (1024 products per accumulator); the chunk loop
// is the outer one, so every slot of a chunk reads the same few K tiles of
// all slices while they are still in L2 (the int64 total is a plain sum, so
// the order of the chunk drains does not change it).
// Parameters and operand maps of global unit u: the launch's own (single
// problem) or, in a grouped launch, those of the problem that owns u.
template <bool kGrouped>
__device__ __forceinline__ const SgParams &unit_params(const SgParams &p, const SgGroup &g, int u, int &local,
                                                      int &mol) {
  if (!kGrouped) {
    local = u;
    mol = 0;
    return p;
  }
  int lo = 0, hi = g.nmol - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.unit_off[mid] <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  mol = lo;
  local = u - g.unit_off[lo];
  return g.params[lo];
}

template <int kMode, bool kGrouped, bool kPair>
__global__ void __launch_bounds__(kThreads, 1)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_b,
                      const SgParams p, const SgGroup grp) {
  constexpr int NS = kPair ? kStagesP : (kMode == kModeMod ? kStagesM : kStages);
  constexpr int SB = (kPair || kMode == kModeMod) ? kStageBytesP : kStageBytes;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + NS * SB);
  uint64_t *empty = full + NS;
  uint64_t *acc_full = empty + NS;
  uint64_t *acc_empty = acc_full + kAccBufs;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + kAccBufs);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // CTA pair: rank 0 issues the MMAs of both CTAs; each CTA loads its own A
  // tile and B tile, drains its own TMEM rows and writes its own output tile.
  const int crank = kPair ? (int)cluster_ctarank() : 0;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      // pair: rank 0's full barriers count the bytes of both CTAs' copies
      // (rank 0's producer expects them all); rank 1's are not used
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < kAccBufs; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], kPair ? 2 * kEpiWarps : kEpiWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    if (kPair) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  // the other CTA's arrivals and commits may target this CTA's barriers from now on
  if (kPair) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int total_units = kGrouped ? grp.total : (kPair ? p.npairs : p.nunits);
  const int first_unit = kPair ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int unit_stride = kPair ? (int)(gridDim.x >> 1) : (int)gridDim.x;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsLow));
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      const uint32_t full0 = kPair ? peer_addr(full, 0) : 0u;
      for (int u = first_unit; u < total_units && ok; u += unit_stride) {
        int lu, mol;
        const SgParams &q = unit_params<kGrouped>(p, grp, u, lu, mol);
        const Unit w = kPair ? decode_pair(q, lu, crank) : decode_unit(q, lu);
        const CUtensorMap *ma = kGrouped ? &grp.maps[2 * mol] : &tmap_a;
        const CUtensorMap *mb = kGrouped ? &grp.maps[2 * mol + 1] : &tmap_b;
        const int nch = num_chunks(w.ktiles);
        for (int c = 0; c < nch && ok; ++c) {
          const int kb = chunk_begin(w.ktiles, nch, c), ke = chunk_begin(w.ktiles, nch, c + 1);
          for (int t = 0; t < w.s && ok; ++t) {
            for (int u0 = 0; u0 <= w.s - 1 - t && ok; u0 += 2) {
              const bool two = u0 + 1 <= w.s - 1 - t;
              for (int kt = kb; kt < ke; ++kt) {
                const uint32_t stage = it % NS;
                const uint32_t ph = (it / NS) & 1;
                if (!wait_bounded<kPair>(&empty[stage], ph ^ 1, abort_flag, p.status)) {
                  ok = false;
                  break;
                }
                uint8_t *sa = smem + stage * SB;
                uint8_t *sb = sa + kTileBytes;
                const int kc = ktile_of(w, kt) * kKTile;
                if (kPair) {
                  // rank r holds B_{u0+r}; a single pair leaves rank 1's B
                  // rows unloaded (their MMA columns 128-255 are not read).
                  // Both CTAs' copies complete on rank 0's barrier.
                  const bool loadb = two || crank == 0;
                  const uint32_t fb = full0 + stage * (uint32_t)sizeof(uint64_t);
                  if (crank == 0) mbar_expect_tx(&full[stage], two ? 4 * kTileBytes : 3 * kTileBytes);
                  tma_load_3d_pair(sa, ma, fb, kc, w.m0, w.az0 + t * w.azs);
                  if (loadb) tma_load_3d_pair(sb, mb, fb, kc, w.n0, w.bz0 + (u0 + crank) * w.bzs);
                } else {
                  mbar_expect_tx(&full[stage], two ? 3 * kTileBytes : 2 * kTileBytes);
                  tma_load_3d(sa, ma, &full[stage], kc, w.m0, w.az0 + t * w.azs);
                  tma_load_3d(sb, mb, &full[stage], kc, w.n0, w.bz0 + u0 * w.bzs);
                  if (two) tma_load_3d(sb + kTileBytes, mb, &full[stage], kc, w.n0, w.bz0 + (u0 + 1) * w.bzs);
                }
                ++it;
              }
            }
          }
        }
      }
      if (!ok && crank == 0) {
        // let the copies already issued land before the CTA goes away
        const uint32_t first = it > (uint32_t)NS ? it - NS : 0u;
        for (uint32_t j = first; j < it; ++j)
          wait_bounded<kPair>(&full[j % NS], (j / NS) & 1, abort_flag, p.status, false);
      } else if (!ok) {
        // pair, rank 1: its copies complete on rank 0's barrier, which this
        // CTA cannot wait on; a copy lands within microseconds, so give the
        // ones in flight a fixed 200 us
        const uint64_t t0 = globaltimer_ns();
        while (globaltimer_ns() - t0 < 200000ull) {
        }
      } else if (kPair) {
        // the MMA commits of the last stages arrive from rank 0: let them
        // land before this CTA can leave
        const uint32_t first = it > (uint32_t)NS ? it - NS : 0u;
        for (uint32_t j = first; j < it; ++j)
          wait_bounded<kPair>(&empty[j % NS], (j / NS) & 1, abort_flag, p.status, false);
      }
    }
  } else if (warp == 1 && kPair && crank != 0) {
    // pair, rank 1: rank 0's thread issues the MMAs of both CTAs
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsLow));
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsLow));
    uint32_t it = 0, qc = 0;
    bool ok = true;
    for (int u = first_unit; u < total_units && ok; u += unit_stride) {
      int lu, mol;
      const SgParams &q = unit_params<kGrouped>(p, grp, u, lu, mol);
      const Unit w = kPair ? decode_pair(q, lu, crank) : decode_unit(q, lu);
      const int nch = num_chunks(w.ktiles);
      for (int c = 0; c < nch && ok; ++c) {
        const int kb = chunk_begin(w.ktiles, nch, c), ke = chunk_begin(w.ktiles, nch, c + 1);
        for (int t = 0; t < w.s && ok; ++t) {
          for (int u0 = 0; u0 <= w.s - 1 - t && ok; u0 += 2) {
            const bool two = u0 + 1 <= w.s - 1 - t;
            const uint32_t idesc = kPair ? kIdescPair : (two ? kIdesc256 : kIdesc128);
            const uint32_t buf = qc % kAccBufs;
            if (!wait_bounded<kPair>(&acc_empty[buf], ((qc / kAccBufs) & 1) ^ 1, abort_flag, p.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            for (int kt = kb; kt < ke; ++kt) {
              const uint32_t stage = it % NS;
              const uint32_t ph = (it / NS) & 1;
              if (!wait_bounded<kPair>(&full[stage], ph, abort_flag, p.status)) {
                ok = false;
                break;
              }
              tc_fence_after();
              if (lane == 0) {
                const uint32_t sa = smem_u32(smem + stage * SB);
                const uint32_t sb = sa + kTileBytes;
                const uint32_t dt = tmem_base + buf * kAccCols;
#pragma unroll
                for (int k = 0; k < kKTile / 16; ++k) {
                  if (kPair)
                    umma_bf16_pair(dt, sw128_desc(sa + k * 32), sw128_desc(sb + k * 32), idesc,
                                   (kt > kb || k > 0) ? 1u : 0u);
                  else
                    umma_bf16(dt, sw128_desc(sa + k * 32), sw128_desc(sb + k * 32), idesc,
                              (kt > kb || k > 0) ? 1u : 0u);
                }
                if (kPair)
                  umma_commit_pair(&empty[stage]);
                else
                  umma_commit(&empty[stage]);
              }
              __syncwarp();
              ++it;
            }
            if (!ok) break;
            if (lane == 0) {
              if (kPair)
                umma_commit_pair(&acc_full[buf]);
              else
                umma_commit(&acc_full[buf]);
            }
            __syncwarp();
            ++qc;
          }
        }
      }
    }
    if (!ok && lane == 0) {
      // wait for the MMAs already issued before the TMEM is released
      uint64_t *done = &acc_full[qc % kAccBufs];
      if (kPair)
        umma_commit_pair(done);
      else
        umma_commit(done);
      wait_bounded<kPair>(done, (qc / kAccBufs) & 1, abort_flag, p.status, false);
    }
    __syncwarp();
  } else if (warp < kEpiWarp0) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsLow));
  } else {
    // ------------------------------------------------------------ epilogue
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsHigh));
    const int quad = warp & 3;
    const int half = (warp - kEpiWarp0) >> 2;
    const int row = quad * 32 + lane;
    const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 64);
    // the buffer is handed back to the MMA issuer: this CTA's, or rank 0's in a pair
    const uint32_t acc_empty0 = kPair ? peer_addr(acc_empty, 0) : 0u;
    long long R[64];
    uint32_t qc = 0;
    bool ok = true;
    for (int u = first_unit; u < total_units && ok; u += unit_stride) {
      int lu, mol;
      const SgParams &q = unit_params<kGrouped>(p, grp, u, lu, mol);
      const Unit w = kPair ? decode_pair(q, lu, crank) : decode_unit(q, lu);
      const int s = w.s;
      const int T = kMode == kModeRaw ? 0 : q.shiftT[s];
      const int m = w.m0 + row;
      const int n_base = w.n0 + half * 64;
      int ea_m = 0;
      if ((kMode == kModeX || kMode == kModeGemm) && m < q.m_valid) ea_m = q.ea[m];
      const int kexp_base = -14 - 8 * (s - 1) + T;
#pragma unroll
      for (int j = 0; j < 64; ++j) R[j] = 0;
      const int nch = num_chunks(w.ktiles);
      for (int c = 0; c < nch && ok; ++c) {
        for (int t = 0; t < s && ok; ++t) {
          for (int u0 = 0; u0 <= s - 1 - t && ok; u0 += 2) {
            const bool two = u0 + 1 <= s - 1 - t;
            const int g0 = t + u0;
            const int sh0 = kMode == kModeRaw ? 0 : 8 * (s - 1 - g0) - T;
            const int sh1 = sh0 - 8;
            const uint32_t buf = qc % kAccBufs;
            if (!wait_bounded<kPair>(&acc_full[buf], (qc / kAccBufs) & 1, abort_flag, p.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t acc = lane_base + buf * kAccCols;
            // 16 columns of each half at a time keeps 32 loaded values live
            // next to the 64 int64 totals (no register spills)
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              uint32_t a0[16], b0[16];
              tmem_ld16(acc + qq * 16, a0);
              if (two) tmem_ld16(acc + 128 + qq * 16, b0);
              tmem_wait_ld();
              if (qq == 3) {
                // the chunk is in registers: hand the buffer back to the MMA warp
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                  if (kPair)
                    mbar_arrive_remote(acc_empty0 + buf * (uint32_t)sizeof(uint64_t));
                  else
                    mbar_arrive(&acc_empty[buf]);
                }
              }
              if constexpr (kMode == kModeRaw) {
                if (m < q.m_valid) {
#pragma unroll
                  for (int j = 0; j < 16; ++j) {
                    const int n = n_base + qq * 16 + j;
                    if (n >= q.n_valid) continue;
                    const int v0 = __float2int_rz(__uint_as_float(a0[j]));
                    q.raw[((long long)g0 * q.n_valid + n) * q.m_valid + m] += (long long)v0;
                    if (two) {
                      const int v1 = __float2int_rz(__uint_as_float(b0[j]));
                      q.raw[((long long)(g0 + 1) * q.n_valid + n) * q.m_valid + m] += (long long)v1;
                    }
                  }
                }
              } else if (two && sh1 >= 0 && sh0 <= 30) {
                // both weights are powers of two that fit a 32-bit multiplier:
                // one widening multiply-add per value (the int64 total is exact,
                // so the sums modulo 2^64 are the sums)
                const int p0 = 1 << sh0, p1 = 1 << sh1;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  R[qq * 16 + j] = mad_pow2(__float2int_rz(__uint_as_float(a0[j])), p0, R[qq * 16 + j]);
                  R[qq * 16 + j] = mad_pow2(__float2int_rz(__uint_as_float(b0[j])), p1, R[qq * 16 + j]);
                }
              } else if (two && sh0 >= 32 && sh1 >= 0 && sh1 <= 30) {
                // the leading pair's weight is 2^32 or more: it adds to the high word
                const int p1 = 1 << sh1;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  R[qq * 16 + j] = add_high(__float2int_rz(__uint_as_float(a0[j])), sh0 - 32, R[qq * 16 + j]);
                  R[qq * 16 + j] = mad_pow2(__float2int_rz(__uint_as_float(b0[j])), p1, R[qq * 16 + j]);
                }
              } else if (two && sh1 >= 0) {
                // both weights are non-negative powers of two, 2^8 apart:
                // v0 2^sh0 + v1 2^sh1 = (v0 2^8 + v1) 2^sh1, exact in int64
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  const int v0 = __float2int_rz(__uint_as_float(a0[j]));
                  const int v1 = __float2int_rz(__uint_as_float(b0[j]));
                  const long long w2 = ((long long)v0 << 8) + (long long)v1;
                  R[qq * 16 + j] += w2 << sh1;
                }
              } else if (!two && sh0 >= 0 && sh0 <= 30) {
                const int p0 = 1 << sh0;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  R[qq * 16 + j] = mad_pow2(__float2int_rz(__uint_as_float(a0[j])), p0, R[qq * 16 + j]);
              } else if (!two && sh0 >= 32) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  R[qq * 16 + j] = add_high(__float2int_rz(__uint_as_float(a0[j])), sh0 - 32, R[qq * 16 + j]);
              } else if (!two && sh0 >= 0) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  const int v0 = __float2int_rz(__uint_as_float(a0[j]));
                  R[qq * 16 + j] += (long long)v0 << sh0;
                }
              } else {
                // some low-order group falls below the kept bits (T > 0): rounded shifts
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  const int v0 = __float2int_rz(__uint_as_float(a0[j]));
                  long long add = weigh(v0, sh0);
                  if (two) add += weigh(__float2int_rz(__uint_as_float(b0[j])), sh1);
                  R[qq * 16 + j] += add;
                }
              }
            }
            ++qc;
          }
        }
      }
      if (ok && kMode != kModeRaw) store64<kMode>(q, w, m, n_base, R, kexp_base, ea_m);
      if constexpr (kMode == kModeX || kMode == kModeXs) {
        if (ok && q.rowE) record_row_bound<kMode>(q, m, n_base, R, kexp_base, lane);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // neither CTA of a pair frees its TMEM or leaves while the other may still
  // use its barriers, shared memory or accumulators
  if (kPair) cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    if (kPair)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                   : "memory");
  }
}

// Failure-path self-test of the bounded wait: one thread waits, through the
// pipeline's own wait routine, on an mbarrier that expects an arrival nobody
// makes.  The wait gives up after limit_ns, raises the CTA's abort flag and
// the status bit, and the kernel returns normally (no trap, no fault).
__global__ void wait_selftest_kernel(int *status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!wait_bounded<false>(&bar, 0, &abort_flag, status, true, limit_ns) && !abort_flag) atomicOr(status, 2);
  }
}

typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                    CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                    CUtensorMapFloatOOBfill);

PFN_encodeTiled get_encode_fn() {
  static PFN_encodeTiled fn = nullptr;
  if (!fn) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled>(ptr);
  }
  return fn;
}

}  // namespace

bool make_tmap_bf16(CUtensorMap *map, const void *base, long long k, long long rows, long long planes,
                    long long row_stride_elems, long long plane_stride_elems) {
  PFN_encodeTiled enc = get_encode_fn();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (row_stride_elems * 2) % 16 || (plane_stride_elems * 2) % 16)
    return false;
  cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(row_stride_elems * 2), (cuuint64_t)(plane_stride_elems * 2)};
  cuuint32_t box[3] = {(cuuint32_t)kKTile, (cuuint32_t)kTile, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Truncation T of the int64 fixed-point sum: |R| <= sum_g (g+1) K 2^14
// 2^(8(s-1-g)) must stay below 2^61 after dropping T low bits.  T = 0 (exact)
// whenever that bound allows it.
int fixed_point_shift(int s, long long k) {
  if (s <= 0) return 0;
  long double bound = 0.0L;
  for (int g = 0; g < s; ++g) bound += (long double)(g + 1) * (long double)k * 16384.0L * ldexpl(1.0L, 8 * (s - 1 - g));
  int bits = 0;
  while (ldexpl(1.0L, bits) < bound) ++bits;
  return bits > 61 ? bits - 61 : 0;
}

cudaError_t launch_wait_selftest(int *status, unsigned long long limit_ns, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(status, limit_ns);
  return cudaGetLastError();
}

int slice_gemm_grid(int nunits) {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  return nunits < nsm ? nunits : nsm;
}

template <int kMode, bool kGrouped>
cudaError_t launch_mode(const SgParams &p, const CUtensorMap &ta, const CUtensorMap &tb, const SgGroup &g, int grid,
                        cudaStream_t st) {
  constexpr int smem = kMode == kModeMod ? kSmemBytesM : kSmemBytes;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(slice_gemm_kernel<kMode, kGrouped, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  slice_gemm_kernel<kMode, kGrouped, false><<<grid, kThreads, smem, st>>>(ta, tb, p, g);
  return cudaGetLastError();
}

// CTA-pair launch: clusters of two CTAs, as many clusters as fit at once
// (at most one per tile pair), persistent over the tile pairs; grouped: the
// tile pairs of several problems (g.total pairs, prefix table in pairs).
template <int kMode, bool kGrouped = false>
cudaError_t launch_pair(const SgParams &p, const CUtensorMap &ta, const CUtensorMap &tb, cudaStream_t st,
                        const SgGroup *grp = nullptr) {
  auto kern = slice_gemm_kernel<kMode, kGrouped, true>;
  static int max_clusters = 0;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = kSmemBytesP;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (!max_clusters) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytesP);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(2 * (unsigned)(slice_gemm_grid(1 << 30) / 2), 1, 1);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = slice_gemm_grid(1 << 30) / 2;
    }
    max_clusters = n > 0 ? n : 1;
  }
  const int np = kGrouped ? grp->total : p.npairs;
  const int nc = np < max_clusters ? np : max_clusters;
  cfg.gridDim = dim3(2 * (unsigned)nc, 1, 1);
  SgGroup g;
  std::memset(&g, 0, sizeof(g));
  if (kGrouped) g = *grp;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ta, tb, p, g);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

long long slice_gemm_pairs(const SgParams &p) {
  if (p.layout == kLayoutKPart) {
    const long long nt = p.nt_m, na = (nt + 1) / 2;
    return na * (nt - na + 1) * p.nblk * p.nsplit;
  }
  if (p.layout == kLayoutXs) return (long long)((p.nt_m + 1) / 2) * p.nt_n;  // many m tiles: one may idle
  if (p.nt_m % 2) return 0;
  return (long long)(p.nt_m / 2) * p.nt_n;
}

// Whether a launch runs in CTA-pair mode.  p.pair: 0 never; 1 the first
// exchange GEMM (every tile pair is useful there); 2 also the second, whose
// pairs recompute one lower tile per pair of tile rows.
static bool use_pairs(const SgParams &p) {
  if (p.pair == 0 || (p.mode != kModeX && p.mode != kModeXs && p.mode != kModeKPart)) return false;
  const long long np = slice_gemm_pairs(p);
  if (np <= 0 || np > (1ll << 30)) return false;
  return p.mode == kModeX || p.mode == kModeXs || p.pair == 2;
}

cudaError_t launch_slice_gemm(const SgParams &p, const CUtensorMap &ta, const CUtensorMap &tb, cudaStream_t st) {
  if (p.nunits <= 0) return cudaSuccess;
  if (use_pairs(p)) {
    SgParams q = p;
    q.npairs = (int)slice_gemm_pairs(p);
    if (p.mode == kModeX) return launch_pair<kModeX>(q, ta, tb, st);
    if (p.mode == kModeXs) return launch_pair<kModeXs>(q, ta, tb, st);
    return launch_pair<kModeKPart>(q, ta, tb, st);
  }
  SgGroup g;
  std::memset(&g, 0, sizeof(g));
  const int grid = slice_gemm_grid(p.nunits);
  switch (p.mode) {
    case kModeX: return launch_mode<kModeX, false>(p, ta, tb, g, grid, st);
    case kModeKPart: return launch_mode<kModeKPart, false>(p, ta, tb, g, grid, st);
    case kModeRaw: return launch_mode<kModeRaw, false>(p, ta, tb, g, grid, st);
    case kModeGemm: return launch_mode<kModeGemm, false>(p, ta, tb, g, grid, st);
    case kModeXs: return launch_mode<kModeXs, false>(p, ta, tb, g, grid, st);
    case kModeMod: return launch_mode<kModeMod, false>(p, ta, tb, g, grid, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_slice_gemm_grouped(int mode, const SgGroup &g, int *status, int grid, cudaStream_t st,
                                      bool pairs) {
  if (g.total <= 0) return cudaSuccess;
  SgParams p;
  std::memset(&p, 0, sizeof(p));
  p.status = status;
  CUtensorMap dummy;
  std::memset(&dummy, 0, sizeof(dummy));
  if (pairs) {
    if (mode == kModeXs) return launch_pair<kModeXs, true>(p, dummy, dummy, st, &g);
    return cudaErrorInvalidValue;
  }
  const int full_grid = slice_gemm_grid(g.total);
  const int gsz = grid > 0 && grid < full_grid ? grid : full_grid;
  switch (mode) {
    case kModeX: return launch_mode<kModeX, true>(p, dummy, dummy, g, gsz, st);
    case kModeKPart: return launch_mode<kModeKPart, true>(p, dummy, dummy, g, gsz, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace df
