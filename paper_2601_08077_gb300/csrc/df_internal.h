// Internal declarations of libdf: the context, the kernel launchers and the
// slice-GEMM work description.  Not part of the public ABI (include/df.h).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cstdint>
#include <vector>

#include "../../include/df.h"
#include "df_device.cuh"

namespace df {

constexpr int kTile = 128;       // output tile edge of the slice GEMM
constexpr int kKTile = 64;       // K elements per pipeline stage (128 bytes of bf16)
constexpr int kMaxChunk = 1024;  // products per exact FP32 accumulation chunk

// Epilogue modes of the slice GEMM.
enum SgMode : int {
  kModeX = 0,       // first exchange GEMM: int64 sums R[n*ld + m] of X^T = C^T B^T (the X split rounds them)
  kModeKPart = 1,   // second exchange GEMM: int64 fixed-point partial per (block, K split),
                    // raw[part*blk + n*ld + m] (the reduce scales and sums them)
  kModeRaw = 2,     // exact S_g per group: raw[(g*n_valid + n)*m_valid + m]
  kModeGemm = 3,    // generic emulated product: out[m*ld + n]
  kModeXs = 4,      // first exchange GEMM with swapped operands (rows (P, mu) on the A side):
                    // int64 sums R[m*ld + n], the same X layout as kModeX
  kModeMod = 5,     // CRT variant: the exact sum of one modulus plane reduced modulo that
                    // modulus, one byte each: out8[plane*out_blk + m*ld + n]
};

// How the persistent kernel turns a unit index into a tile.
enum SgLayout : int {
  kLayoutGrid = 0,   // u -> (m_tile = u % nt_m, n_tile = u / nt_m), planes az = t, bz = t
  kLayoutX = 1,      // first exchange GEMM: n rows are (P, mu); block = n0 / (128 nao)
  kLayoutKPart = 2,  // second exchange GEMM: u -> (upper tile pair, block)
  kLayoutXs = 3,     // first exchange GEMM, swapped: m rows are (P, mu); block = m0 / (128 nao)
  kLayoutCrt = 4,    // CRT variant: u -> (plane = u / (nt_m nt_n), grid tile), planes az = bz = plane
};

constexpr int kCrtMaxModuli = 16;

// Blocks of the density-change reduction ||D - D_prev||_F (df_build_J).
constexpr int kDensityChangeBlocks = 152;

// Row splits give a whole 256-thread block to each row at least this wide
// (fewer, longer rows: the second exchange GEMM's operands), else a warp.
constexpr int kWideRow = 2048;

struct SgParams {
  int layout, mode;
  int nunits;
  int nt_m, nt_n;           // tiles along m and n
  int m_valid, n_valid;     // rows of the A side and of the B side that exist
  int ktiles;               // K tiles (64 wide) for kLayoutGrid / kLayoutX
  int s_fixed;              // slice count for kLayoutGrid
  int nao, nocc, nblk, naux;
  int nsplit;               // K splits per block (kLayoutKPart)
  const int *s_blk;         // per-block slice counts (kLayoutX, kLayoutKPart)
  int shiftT[9];            // truncation T of the fixed-point sum, indexed by s (0..8)
  const int *ea;            // A-side row exponents
  const int *eb;            // B-side row exponents
  long long out_ld;
  long long out_blk;
  double *out;
  long long *raw;
  int *status;              // device status word (DF_ERR_TIMEOUT bits)
  // CTA-pair mode: two CTAs of a cluster take two tiles that share their
  // B-side operand; each CTA loads its own A tile and one of the two stacked
  // B tiles into its own shared memory (both copies complete on the first
  // CTA's barrier), and one M = 256 MMA reads both CTAs' tiles.  Work is
  // then counted in tile pairs (npairs); the host sets both.
  int pair;
  int npairs;
  int crt_mod[kCrtMaxModuli];  // kModeMod: the modulus of each plane
  // first exchange GEMM on a screened (block-sparse) B: per 128-row tile of
  // B's (P, mu) rows, the bit mask of its nonzero 64-wide K tiles (bit k = K
  // tile k, at most 32); null = dense
  const uint32_t *kmask;
  // first exchange GEMM (kModeX / kModeXs): per (block, mu) row of X, the
  // largest bit-length bound E = bitlen(|R|) + k over the row's nonzero exact
  // sums R (|R 2^k| < 2^E), atomically maxed; the X split takes it as its
  // exponent guess and so reads R once.  Reset to kRowBoundNone before the
  // launch; null = not recorded.
  int *rowE;
};

// "No nonzero element yet" in a row bound (the byte 0x80 repeated, so a
// memset resets it); below every real bound.
constexpr int kRowBoundNone = (int)0x80808080;

// Tile pairs of a launch in CTA-pair mode (0 = the layout has no pairing):
// kLayoutGrid / kLayoutX pair m tiles 2a, 2a+1 of one n tile (nt_m even);
// kLayoutKPart pairs m tiles 2a, 2a+1 of n tile j >= 2a per (block, split).
long long slice_gemm_pairs(const SgParams &p);

// A grouped launch: the work units of several problems (molecules) in one
// persistent launch.  Problem i owns units [unit_off[i], unit_off[i+1]); its
// parameters are params[i] and its operand tensor maps maps[2i] (A side) and
// maps[2i+1] (B side), all in device memory (maps 64-byte aligned).
struct SgGroup {
  const SgParams *params;
  const CUtensorMap *maps;
  const int *unit_off;
  int nmol;
  int total;
};

struct Ctx;

// Scratch of the stand-alone emulated-GEMM entry points: stream-ordered
// allocations from the device's default pool, whose release threshold is
// raised once so that repeated calls reuse the memory instead of mapping it
// again (it stays reserved by the process until cudaDeviceReset).
inline cudaError_t scratch_malloc(void **p, size_t bytes, cudaStream_t st) {
  static bool kept[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !kept[dev]) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    kept[dev] = true;
  }
  return cudaMallocAsync(p, bytes, st);
}

// Kernel launchers (split.cu, slicegemm.cu, coulomb.cu).
cudaError_t launch_split_rows_bf16(const double *A, long long rows, int cols, long long ld, int nslices,
                                   int *exps, uint16_t *digits, long long dld, long long plane_stride,
                                   cudaStream_t st, const int *perm = nullptr, int group = 1);
cudaError_t launch_split_rows_int8(const double *A, int rows, int cols, int ld, int nslices, int *exps,
                                   int8_t *digits, cudaStream_t st);
cudaError_t launch_split_cols_bf16(const double *C, int nrows, int ncols, int nslices, int *exps,
                                   uint16_t *digits, long long dld, long long plane_stride, cudaStream_t st);
struct ShiftTable {
  int v[9];
};
// R: the first GEMM's int64 sums (kModeX); X = fl64(R 2^k) is formed here with
// the first GEMM's exponents eB (rows (P, mu)), eC (orbitals), slices s_blk and
// truncation table T1, then split per (block, mu).  rowE: the first GEMM's
// per-row bound (SgParams::rowE) when it recorded one, else null.
cudaError_t launch_split_xblocks(const long long *R, int naux, int nao, int nocc, int nslices, const int *eB,
                                 const int *eC, const int *s_blk, const ShiftTable &T1, const int *rowE, int *eX,
                                 uint16_t *Xd, long long kb_ld, int nblk, cudaStream_t st);
cudaError_t launch_kpart_reduce(const long long *Rp, const int *eX, const int *s_blk, ShiftTable T, int nao,
                                int nblk, int nsplit, double *K, cudaStream_t st);

// Encode a 3D bf16 tensor map {k, rows, planes} with a 64 x 128 x 1 box, 128B swizzle.
bool make_tmap_bf16(CUtensorMap *map, const void *base, long long k, long long rows, long long planes,
                    long long row_stride_elems, long long plane_stride_elems);

cudaError_t launch_slice_gemm(const SgParams &p, const CUtensorMap &ta, const CUtensorMap &tb,
                              cudaStream_t st);
// Grouped launch; `mode` is shared by all problems, `grid` CTAs (0 = one per SM).
// pairs: CTA-pair launch over tile pairs (kModeXs only; unit_off and total
// count tile pairs, every problem's npairs set).
cudaError_t launch_slice_gemm_grouped(int mode, const SgGroup &g, int *status, int grid, cudaStream_t st,
                                      bool pairs = false);
int slice_gemm_grid(int nunits);
// One-thread kernel whose bounded wait on a never-completed mbarrier runs out
// after limit_ns and sets bit 0 of *status (bit 1: it returned without the
// abort path, which would be a defect).
cudaError_t launch_wait_selftest(int *status, unsigned long long limit_ns, cudaStream_t st);
int fixed_point_shift(int s, long long k);

// mask_mu (optional, block-sparse B): per mu, bit c set when some B_P mu nu
// with nu in [64c, 64c + 64) is nonzero; null = dense.
// packed: B holds per P the upper triangle row by row ([naux][nao (nao + 1) / 2]).
// work (optional): a zeroed item counter; then `grid` CTAs take the items from
// it (a short grid sharing the SMs with a concurrent kernel), else one CTA
// per item.  Either way every rho_P and J_mn is summed in the same order.
// rows: rho in the row-by-row order of a B with zero chunks (taken whenever
// mask_mu is given), else in row-pair order; the order is the B's, so a
// screened B gives the same bits with and without its masks.
cudaError_t launch_rho(const double *B, const double *D, int naux, int nao, double *rho, cudaStream_t st,
                       const uint32_t *mask_mu = nullptr, bool packed = false, int *work = nullptr, int grid = 0,
                       bool rows = false);
cudaError_t launch_coulomb(const double *B, const double *rho, int naux, int nao, double *J, cudaStream_t st,
                           const uint32_t *mask_mu = nullptr, bool packed = false, int *work = nullptr,
                           int grid = 0);
// The masks of a packed B (pair flags through stream-ordered scratch of nao (nao + 1) / 2 bytes).
cudaError_t launch_pair_masks_packed(const double *Bp, int naux, int nao, uint32_t *mask_mu, uint32_t *mask_tile,
                                     cudaStream_t st);
// Dense B_P, P = P0 .. P0 + nP - 1, into out [nP][nao][nao] from a packed B.
cudaError_t launch_unpack(const double *Bp, int P0, int nP, int nao, double *out, cudaStream_t st);
// Digits of B from its packed layout (rows (P', mu) as launch_split_rows_bf16 writes them).
cudaError_t launch_split_rows_packed(const double *Bp, int naux, int nao, int nslices, int *exps, uint16_t *digits,
                                     long long dld, long long plane_stride, const int *perm, cudaStream_t st);
// Sets *flag (zeroed first) when some B_P of B [naux][nao][nao] is not exactly
// symmetric.
cudaError_t launch_symmetry_check(const double *B, int naux, int nao, int *flag, cudaStream_t st);
// The masks of a screened B: mask_mu as above (nao <= 2048) and, per
// 128-row tile of the (P, mu) rows, the OR of its rows' mu masks.
cudaError_t launch_pair_masks(const double *B, int naux, int nao, uint32_t *mask_mu, uint32_t *mask_tile,
                              cudaStream_t st);
cudaError_t launch_energy(const double *D, const double *J, const double *K, const double *rho, int nao,
                          int naux, double *partials, double *E_dev, cudaStream_t st);

}  // namespace df
