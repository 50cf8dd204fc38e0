// The context behind the opaque df_ctx handle of the C ABI (internal).
#pragma once
#include <utility>
#include <vector>

#include "df_internal.h"

struct df_ctx {
  int nao = 0, naux = 0, nocc_max = 0, s_max = 0, nblk = 0;
  long long ld_nao = 0;    // row stride (elements) of the B and C digit rows
  long long kb_ld_max = 0; // row stride bound of the X digit rows
  const double *B = nullptr;  // dense [naux][nao][nao], or packed [naux][nao (nao + 1) / 2]
  bool packed = false;
  bool ready = false;
  uint16_t *Bd = nullptr;
  int *eB = nullptr;
  uint16_t *Cd = nullptr;
  int *eC = nullptr;
  double *X = nullptr;  // emulated path: the first GEMM's int64 sums (same size); FP64 path: X^T
  uint16_t *Xd = nullptr;
  int *eX = nullptr;
  int *rowE = nullptr;      // [nblk][nao] the first GEMM's bound on each X row's exponent
  long long *Rp = nullptr;  // int64 partials of the second GEMM [nblk][nsplit][nao][nao]
  int nsplit = 1;
  double *rho = nullptr;
  // df_build_JK: rho and J on a high-priority internal stream beside the X
  // split, from short grids of jk_ctas CTAs per SM taking items from the two
  // counters jk_work (0: everything in the caller's stream, in order)
  int *jk_work = nullptr;
  int jk_ctas = 4;
  int nsm = 0;
  cudaStream_t jk_stream = nullptr;
  cudaEvent_t jk_fork = nullptr, jk_join = nullptr;
  double *epart = nullptr;
  double *E = nullptr;
  int *sblk = nullptr;      // device per-block slice counts
  int *sblk_host = nullptr; // pinned mirror of the last upload
  int *status = nullptr;
  double *bstats = nullptr;  // static per-block statistics for the predictor's features
  // block sparsity of a screened B (set up by df_setup): per mu the mask of
  // nonzero 64-wide nu chunks, per 128-row tile of (P, mu) rows the OR of its
  // rows' masks; used only when some chunk is zero (sparse)
  uint32_t *mask_mu = nullptr;
  uint32_t *mask_tile = nullptr;
  bool sparse = false;
  int sparse_opt = 1;        // DF_OPT_SPARSE: 0 never use the masks, 1 when some chunk is zero
  double frac_ktiles = 1.0;  // nonzero K tiles of the first GEMM's row tiles
  double frac_chunks = 1.0;  // nonzero (mu, 64-wide nu chunk) pairs of the upper triangle
  int *perm = nullptr;       // exchange-path order of the auxiliary functions (P' -> P), or null
  std::vector<int> perm_h;   // host copy of perm (empty: natural order)
  int64_t bytes = 0;
  df_status last = DF_OK;
  cublasHandle_t cublas = nullptr;
  void *cusolver = nullptr;  // cusolverDnHandle_t, created by df_setup_integrals
  // per-phase event timing
  bool profiling = false;
  int pair_mode = 1;  // DF_OPT_CLUSTER_PAIRS
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[DF_NPHASES];
  std::vector<cudaEvent_t> pool;
  // adaptive controller (Section 3.2)
  int level = 4, iter = 0, fp64_from = -1, level0_slices = 0;
  double E_prev = 0.0;
  double dE_last = 1.0;      // last relative energy change seen by df_adaptive_next (1 before any)
  // density change between successive df_build_J calls (a predictor feature)
  double *Dprev = nullptr;   // [nao][nao] the density of the last df_build_J
  double *dD = nullptr;      // device scalar ||D - D_prev||_F (1 before any previous density)
  double *dD_part = nullptr; // partial sums of the reduction
  bool have_Dprev = false;
  // learned slice counts (df_set_predictor; the network's kernels live in mlp.cu)
  df_mlp *pred = nullptr;
  float min_conf = 0.6f;
  float *lF = nullptr;       // [nblk][16] features
  float *lprobs = nullptr;   // [nblk][8] class probabilities
  int *lpick = nullptr;      // [2 nblk] picked counts, low-confidence flags
  int *lexp = nullptr;       // [2 nblk + 1] per block max eX, max eB; then max eC
  int *lhost = nullptr;      // pinned mirror of lpick / lexp
};


namespace df {
// Upload per-block slice counts to the context if they changed (synchronises
// the stream when they did; not allowed during stream capture).
df_status ctx_upload_slices(df_ctx *c, const int *sb, cudaStream_t st);
// Parameters and operand maps of the two exchange GEMMs of a context.
// swap: 0 orbitals on the MMA's M side; 1 (single problem) the (P, mu)-rows-
// on-M layout when CTA pairs are on, nocc <= 128 and nao is even; 2 (grouped,
// one slice count per problem, so a pair may straddle two blocks) that layout
// whenever nocc <= 128.
bool gemm1_setup(df_ctx *c, int nocc, SgParams &p, CUtensorMap &ta, CUtensorMap &tb, int swap = 1);
bool gemm2_setup(df_ctx *c, int nocc, int nsplit, SgParams &q2, CUtensorMap &tx);
long long xdigit_ld(int nocc);
// The sparsity masks to use (null: run dense).
inline const uint32_t *use_mask_mu(const df_ctx *c) { return c->sparse && c->sparse_opt ? c->mask_mu : nullptr; }
inline const uint32_t *use_mask_tile(const df_ctx *c) { return c->sparse && c->sparse_opt ? c->mask_tile : nullptr; }
// The two halves of an emulated exchange build with per-block counts sb:
// the front uploads sb, splits C into c_planes digit planes (>= max sb), runs
// the first GEMM and the X split; the back runs the second GEMM and the
// reduce into K.  Both asynchronous on st.
// after_gemm1 (optional): an event recorded in st right after the first GEMM.
df_status k_front(df_ctx *c, const double *C, int nocc, const int *sb, int c_planes, cudaStream_t st,
                  cudaEvent_t after_gemm1 = nullptr);
df_status k_back(df_ctx *c, int nocc, double *K, cudaStream_t st);
// The slice count run at a Table 1 level under the context's controller
// settings (0 = native FP64).
int level_count(const df_ctx *c, int level);
// The learned-mode exchange build (mlp.cu): predicted per-block counts for the
// context's current level, checked against the level's error bound.
df_status build_K_learned(df_ctx *c, const double *C, int nocc, double *K, df_kstats *stats, cudaStream_t st);
// Launch of ||D - D_prev||_F into c->dD (1 when there is no previous density)
// and the copy D -> D_prev (coulomb.cu).
cudaError_t launch_density_change(const double *D, double *Dprev, bool have_prev, long long n2, double *part,
                                  double *out, cudaStream_t st);
}  // namespace df
