/*
 * libdf: GB300-native adaptive-precision density fitting (C ABI).
 *
 * The hot path of arXiv 2601.08077 ("Accelerating Density Fitting with
 * Adaptive-precision and 8-bit Integer on AI Accelerators"):
 *
 *   Coulomb  (Section 2.1, Eqs. df-j-1, df-j-2):  rho_P = sum_mn B_Pmn D_mn,
 *                                                 J_mn  = sum_P B_Pmn rho_P      (FP64)
 *   Exchange (Section 2.1, Eqs. df-k-1, df-k-2):  X_Pmi = sum_n B_Pmn C_ni,
 *                                                 K_mn  = sum_Pi X_Pmi X_Pni
 *   with both exchange contractions run as FP64-emulating GEMMs over s INT8
 *   slices (Section 3.2), blocked over 128 auxiliary functions
 *   (Section 3.3, Eqs. df-k-blk-1/2), and s chosen by the energy-change rule
 *   of Table 1 (Section 3.2) or per block by a learned predictor.
 *
 * Conventions (every entry point):
 *   - Matrices are row-major FP64.  B is [naux][nao][nao], C is [nao][nocc],
 *     D, J and K are [nao][nao], rho is [naux].
 *   - Pointers named *_dev are device pointers owned by the caller; the
 *     library never frees them.  The context owns its own workspaces
 *     (digit planes, exponents, X, partial K blocks), allocated by df_create.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  All calls are asynchronous on that stream unless
 *     stated otherwise.
 *   - Errors: every call returns a df_status.  A context keeps the first
 *     error it saw (df_last_error).  Device-side waits are bounded; a wait
 *     that runs out sets DF_ERR_TIMEOUT in the context's device status word,
 *     which df_sync_status reads.  No call traps or aborts the process.
 */
#ifndef DF_H_
#define DF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DF_OK = 0,
  DF_ERR_ARG = -1,      /* invalid argument (size, pointer, slice count) */
  DF_ERR_CUDA = -2,     /* a CUDA runtime / cuBLAS call failed */
  DF_ERR_OOM = -3,      /* device allocation failed */
  DF_ERR_NOT_PD = -4,   /* metric not positive definite */
  DF_ERR_TIMEOUT = -5,  /* a bounded device-side wait ran out */
  DF_ERR_TOL = -6,      /* a result missed its tolerance after recompute */
  DF_ERR_STATE = -7,    /* call out of order (e.g. build before setup) */
  DF_ERR_SCRATCH = -8   /* problem too large for df_emulated_gemm_static's fixed scratch */
} df_status;

typedef struct df_ctx df_ctx;

#define DF_S_MAX 8        /* digits per value: 8 x 8 bits >= the 63 bits of RNE(x 2^63) */
#define DF_AUX_BLOCK 128  /* auxiliary functions per block (Section 3.3) */

/* Statistics of one exchange build (host struct, optional). */
typedef struct {
  int nblk;                 /* number of auxiliary blocks */
  int slices[256];          /* slice count used per block (first 256 blocks; 0 = FP64) */
  int recomputed;           /* learned mode: blocks the error-bound check raised and recomputed */
  int fallback;             /* 1 if the build ran in native FP64 */
  int low_confidence;       /* learned mode: blocks that took the level's count for low confidence */
  int level;                /* Table 1 level of an adaptive or learned build; -1 for fixed counts */
  long long slice_pairs;    /* sum over blocks of s_b (s_b + 1) / 2 of the counts used */
  double bound_ratio;       /* learned mode: sum_b beta_b(s_b) / sum_b beta_b(s_level) as run (<= 1) */
} df_kstats;

/* Create a context for one molecule: nao basis functions, naux auxiliary
 * functions, up to nocc_max occupied orbitals, digit planes kept for B up to
 * s_max (1..8).  Allocates all device workspaces on the current device.
 * Returns DF_ERR_OOM if they do not fit. */
df_status df_create(df_ctx **out, int nao, int naux, int nocc_max, int s_max);
void df_destroy(df_ctx *ctx);

/* Attach the DF tensor B (Eq. cderi; device, [naux][nao][nao], caller-owned
 * and kept alive for the context's lifetime) and split it once into s_max
 * INT8 digit planes with one power-of-two exponent per (P, mu) row
 * (Section 3.2).  B is constant over the SCF iterations, so this runs once.
 * Every B_P must be exactly symmetric (B_P mu nu == B_P nu mu bit for bit, as
 * Eq. cderi gives it in exact arithmetic; rho and J read only the upper
 * triangle): the call checks this on the device and returns DF_ERR_ARG
 * otherwise (also for a NaN).  Synchronises `stream`. */
df_status df_setup(df_ctx *ctx, const double *B_dev, void *stream);

/* As df_setup, with the exchange path taking the auxiliary functions in the
 * order perm_host[0..naux-1] (a permutation, new position -> original P):
 * the 128-function blocks, their per-(block, mu) scales and per-block slice
 * counts follow that order.  J and the final K are sums over all P and do
 * not depend on it.  Ordering by magnitude (largest max|B_P| first) gives
 * blocks of similar scale, which the per-block slice counts can exploit.
 * NULL = the natural order.  DF_ERR_ARG if perm_host is not a permutation. */
df_status df_setup_ordered(df_ctx *ctx, const double *B_dev, const int *perm_host, void *stream);

/* As df_setup_ordered, with B given packed: Bp_dev [naux][nao (nao + 1) / 2]
 * holds each B_P's upper triangle row by row (element (mu, nu), nu >= mu, at
 * mu nao - mu (mu - 1) / 2 + nu - mu), the symmetric storage Section 3.3
 * describes, half the bytes of the dense tensor.  Caller-owned and kept alive
 * for the context's lifetime.  rho and J read it directly (bit-identical to a
 * dense B with the same values), the digit planes and the sparsity masks are
 * formed from it, and the native FP64 comparison build unpacks it in chunks
 * of about 1 GB (stream-ordered scratch).  Synchronises `stream`. */
df_status df_setup_packed(df_ctx *ctx, const double *Bp_dev, const int *perm_host, void *stream);

/* As df_setup_ordered, forming B on the device from the integrals
 * (Eq. cderi): B = L^{-1} (P|mu nu) with L L^T = (P|Q) the metric's Cholesky
 * factor.  T_dev [naux][nao][nao] holds (P|mu nu) on entry and B on return
 * (in place; caller-owned and kept alive for the context's lifetime, as in
 * df_setup); V_dev [naux][naux] is the metric (symmetric; read only).  The
 * factorisation (cuSOLVER potrf) and the triangular solve (cuBLAS trsm) are
 * FP64 library steps; every B_P is then made exactly symmetric,
 * (B_P + B_P^T)/2, and split as in df_setup.  perm_host as in
 * df_setup_ordered (NULL = natural order).  Synchronises the stream once (to
 * read the factorisation's status).  Returns DF_ERR_NOT_PD if the metric is
 * not positive definite (T_dev is then unchanged), DF_ERR_OOM if the
 * naux^2 factor workspace cannot be allocated. */
df_status df_setup_integrals(df_ctx *ctx, double *T_dev, const double *V_dev, const int *perm_host, void *stream);

/* Coulomb build in FP64 (Eqs. df-j-1, df-j-2; the paper keeps J in FP64,
 * Section 3.1).  D_dev symmetric [nao][nao]; J_dev [nao][nao] out;
 * rho_dev [naux] out (may be NULL: then an internal buffer is used). */
df_status df_build_J(df_ctx *ctx, const double *D_dev, double *J_dev, double *rho_dev, void *stream);

/* Exchange build (Eqs. df-k-1, df-k-2, blocked as Eqs. df-k-blk-1/2).
 * C_dev [nao][nocc] (nocc <= nocc_max), K_dev [nao][nao] out (full,
 * symmetric).  stats may be NULL.  nslices:
 *   1..8  INT8 emulation with that many slices per operand for every block;
 *   0     native FP64 (cuBLAS DGEMM + DSYRK, the comparison build);
 *   -1    adaptive (Section 3.2, Table 1): the count of the context's current
 *         level, as set by df_adaptive_reset / df_adaptive_next (level 0 runs
 *         native FP64, or the df_adaptive_level0 count);
 *   -2    learned: per-block counts for the current level from the network
 *         attached with df_set_predictor, checked against the level's error
 *         bound (df_set_predictor describes the check); blocks the check
 *         raises are recomputed and counted in stats->recomputed.  At level 0
 *         it runs as -1.  Synchronises `stream` (the predicted counts and the
 *         check's exponents are read on the host); DF_ERR_STATE if no network
 *         is attached. */
df_status df_build_K(df_ctx *ctx, const double *C_dev, int nocc, int nslices, double *K_dev,
                     df_kstats *stats, void *stream);

/* The Coulomb and the exchange build of one density in a single call
 * (Section 2.1, Eqs. df-j-1/2 and df-k-1/2): the results, bit for bit, of
 * df_build_J(ctx, D_dev, J_dev, rho_dev, stream) followed by
 * df_build_K(ctx, C_dev, nocc, nslices, K_dev, stats, stream), with the same
 * arguments, ownership and errors.  For an emulated count (1..8, or -1 at a
 * level that runs slices) the FP64 rho and J kernels run on an internal
 * high-priority stream of the context, forked from `stream` after the first
 * exchange GEMM and joined back before the second: they share the SMs with
 * the X split (rho and J are bound by GB300's FP64 pipe, the X split by HBM
 * and integer work), from short grids of a few CTAs per SM
 * (DF_OPT_JK_OVERLAP).  Native FP64 (0), the learned counts (-2 at a level
 * above 0), a block-sparse B (df_sparsity below 1, with DF_OPT_SPARSE on) and
 * DF_OPT_JK_OVERLAP = 0 run the two builds in order in `stream`.  Calls on
 * one context must not overlap (they share the internal stream and its work
 * counters). */
df_status df_build_JK(df_ctx *ctx, const double *D_dev, const double *C_dev, int nocc, int nslices,
                      double *J_dev, double *rho_dev, double *K_dev, df_kstats *stats, void *stream);

/* Exchange build with one slice count per auxiliary block (host array of
 * ceil(naux/128) entries, each 1..8), given by the caller; no check. */
df_status df_build_K_blocks(df_ctx *ctx, const double *C_dev, int nocc, const int *slices_per_block,
                            double *K_dev, df_kstats *stats, void *stream);

/* Energies (the Coulomb and exchange energies E_J and E_K of Section 3.2, FP64 reductions on the device):
 * E_host[0] = 1/2 tr(D J), E_host[1] = 1/2 rho.rho (second route to E_J),
 * E_host[2] = -1/2 tr(D K).  Synchronises `stream`; rho_dev may be NULL
 * (then the buffer of the last df_build_J is used). */
df_status df_energy(df_ctx *ctx, const double *D_dev, const double *J_dev, const double *K_dev,
                    const double *rho_dev, double *E_host, void *stream);

/* Split rows of an FP64 matrix (device [rows][ld], cols used) into nslices
 * balanced INT8 digits (Section 3.2): exps_dev [rows] (int32) gets the
 * smallest e with max|row| < 127/128 2^e, digits_dev [nslices][rows][cols]
 * (int8) gets d_0..d_{nslices-1} of RNE(A 2^{63-e}).  No context needed. */
df_status df_split_int8(const double *A_dev, int rows, int cols, int ld, int nslices, int32_t *exps_dev,
                        int8_t *digits_dev, void *stream);

/* Exact INT32-range slice-pair products S_g = sum_{t+u=g} A_t B_u^T for
 * g < nslices (Section 3.2) of A (device [M][K]) and B (device [N][K]), both
 * split per row on the device, computed on the tensor cores.  S_dev
 * [nslices][N][M] int64 (note: N-major).  Exps: ea_dev [M], eb_dev [N]
 * (may be NULL).  Test and inspection entry point. */
df_status df_slice_products(const double *A_dev, const double *B_dev, int M, int N, int K, int nslices,
                            int64_t *S_dev, int32_t *ea_dev, int32_t *eb_dev, void *stream);

/* FP64-emulated product out = A B^T (A [M][K], B [N][K], out [M][N], all
 * device, row-major) with nslices INT8 slices per operand (Section 3.2). */
df_status df_emulated_gemm(const double *A_dev, const double *B_dev, int M, int N, int K, int nslices,
                           double *out_dev, void *stream);

/* Same result as df_emulated_gemm, but allocates nothing (the paper has no
 * counterpart: this serves callers that cannot let a library allocate, such
 * as a framework whose memory pool already holds nearly all device memory, or
 * a latency-critical loop that cannot take the synchronisation of
 * cudaMalloc/cudaFree).  Scratch comes from one static 32 MiB device array per
 * GPU; sizes needing more than that return DF_ERR_SCRATCH.  The scratch
 * needed is, with every part rounded up to 256 bytes: a 4-byte status word,
 * 4 M + 4 N bytes of exponents and 2 * nslices * (M + N) * round_up(K, 8)
 * bytes of digit planes; when B_dev == A_dev and N == M (a Gram product) one
 * split serves both operands and the N terms drop out.  The first call on a
 * device looks up the array's device address with that device current: make
 * it before any stream capture.  The address is kept for the process's life,
 * so after a cudaDeviceReset this entry point must not be called on that
 * device again.  Calls share the array, so calls whose GPU work overlaps
 * race.  Synchronises `stream`. */
df_status df_emulated_gemm_static(const double *A_dev, const double *B_dev, int M, int N, int K, int nslices,
                                  double *out_dev, void *stream);

/* CRT variant of the emulated GEMM: Ozaki scheme II (Ozaki, Uchino and
 * Imamura, 2025), the other INT8 emulation Section 2.3 names, computed on the
 * same tensor-core slice GEMM.  Moduli: the integers <= 256 taken greedily
 * downwards, each coprime to the ones before (256, 255, 253, 251, 247, ...),
 * at most DF_CRT_MAX_MODULI.  For K-term sums with n moduli (product M_n) the
 * operands are scaled per row to integers A' = RNE(A 2^(q-1-e)) (e the
 * smallest integer with max|row| < 127/128 2^e) with q the largest width
 * <= 63 such that K 2^(2q-1) < M_n; the exact integer product is rebuilt from
 * its residues by the Chinese remainder theorem and rounded once to FP64. */
#define DF_CRT_MAX_MODULI 16

/* The i-th modulus (0-based); 0 if i is out of range.  Host only. */
int df_crt_modulus(int i);

/* The operand width q for K-term sums with nmod moduli; 0 if K is outside
 * [1, 2^26] or nmod outside [2, 16] or no width >= 2 fits.  Host only. */
int df_crt_operand_bits(long long K, int nmod);

/* The fewest moduli whose width q reaches bits + 1, i.e. the resolution of
 * Table 1's level with m_emu = bits (s = (bits + 1) / 8 slices resolve a row
 * to 2^(e - 8s)); 0 if 16 moduli do not reach it.  Host only. */
int df_crt_moduli_for_bits(long long K, int bits);

/* Inspection entry point: exps_dev [rows] (int32) and the centred residues
 * res_dev [nmod][rows][cols] (int16, in [-floor((m-1)/2), floor(m/2)]) of
 * A' mod m_i for the rows of A (device [rows][ld]) with K = cols. */
df_status df_crt_split_rows(const double *A_dev, int rows, int cols, int ld, int nmod, int32_t *exps_dev,
                            int16_t *res_dev, void *stream);

/* Inspection entry point: y_i = (a_i b_i^T) mod m_i for A (device [M][K]) and
 * B (device [N][K]), Y_dev [nmod][M][N] (uint8), exponents ea_dev [M], eb_dev
 * [N] (may be NULL).  Allocates scratch; synchronises `stream`. */
df_status df_crt_residue_products(const double *A_dev, const double *B_dev, int M, int N, int K, int nmod,
                                  uint8_t *Y_dev, int32_t *ea_dev, int32_t *eb_dev, void *stream);

/* out = A B^T (A [M][K], B [N][K], out [M][N], all device, row-major)
 * emulated with nmod moduli; K <= 2^26.  Allocates scratch (2 nmod (M + N)
 * round_up(K, 8) bytes of residue planes, nmod M round_up(N, 16) bytes of
 * residue products); synchronises `stream`.  DF_ERR_ARG for sizes or a
 * modulus count that admit no width q >= 2. */
df_status df_emulated_gemm_crt(const double *A_dev, const double *B_dev, int M, int N, int K, int nmod,
                               double *out_dev, void *stream);

/* Table 1 (Section 3.2): the emulation level for the next iteration given the
 * relative energy change (>= lower bound of the row); level 0 = FP64. */
int df_level_for(double dE_rel);
/* INT8 splits of a level: 4->3, 3->4, 2->5, 1->6, 0->0 (FP64). */
int df_level_slices(int level);

/* Adaptive controller kept in the context (Section 3.2): call once per
 * iteration with the energy it produced; returns the level for the next
 * iteration.  Iterations 0 and 1 run at level 4; afterwards the level is
 * min(previous, rule(dE_rel)) - precision never drops.  If fp64_from_level
 * >= 0, any level <= it is run as native FP64 (the hardware-specific
 * fallback of Section 3.2). */
df_status df_adaptive_reset(df_ctx *ctx, int fp64_from_level);
/* Slice count run at level 0 (the paper's FP64 level): 0 (default) = native
 * FP64; 7 or 8 = emulation at that many slices (a GB300 variant: its FP64
 * rate is ~40x below the 8-slice emulation, whose K error is ~2e-15). */
df_status df_adaptive_level0(df_ctx *ctx, int nslices);
df_status df_adaptive_next(df_ctx *ctx, double energy, int *level_out, int *nslices_out);

/* Read (and clear) the device status word; synchronises `stream`. */
df_status df_sync_status(df_ctx *ctx, void *stream);

/* Failure-path self-test, without a GPU fault: one thread waits, through the
 * same bounded-wait routine the slice-GEMM pipeline uses, on a barrier that
 * nothing completes; after limit_ms (1 to 10000) the wait gives up, sets the
 * abort flag and the status word, and the kernel returns.  Returns
 * DF_ERR_TIMEOUT when the wait ran out and was reported (the expected
 * result), DF_OK if it was not, DF_ERR_CUDA on a CUDA error.  The CUDA
 * context stays usable.  Synchronises `stream`. */
df_status df_selftest_wait_timeout(int limit_ms, void *stream);
df_status df_last_error(const df_ctx *ctx);
const char *df_strerror(df_status s);

/* ---- Batched builds over many molecules (grouped persistent launches) ----
 * A batch groups n contexts that are already set up (one molecule each, of
 * any size).  df_batch_build_K runs, for all molecules at once: the C
 * splits, ONE persistent launch of the first exchange GEMM over the work
 * units of every molecule, the X splits, ONE persistent launch of the second
 * GEMM, and the reductions (Section 3.3 blocking per molecule, Section 3.2
 * emulation).  With graphs on (the default) the whole sequence is captured
 * once per (nslices, argument pointers) as a CUDA graph and replayed; a NULL
 * stream runs it without a graph.  The per-molecule kernels between the
 * grouped launches (X splits, reductions; in df_batch_build_J each
 * molecule's rho and J) run concurrently on four internal streams that fork
 * from and join back into `stream`, so a call is still ordered with the
 * caller's other work on `stream`.  Pointer arrays are host arrays of device
 * pointers, one per molecule.  The contexts must be distinct (DF_ERR_ARG
 * otherwise: their buffers are written concurrently); the caller keeps them
 * alive. */
typedef struct df_batch df_batch;
df_status df_batch_create(df_batch **out, df_ctx *const *ctxs, int n);
void df_batch_destroy(df_batch *b);
df_status df_batch_set_graphs(df_batch *b, int on);
df_status df_batch_build_K(df_batch *b, const double *const *C_dev, const int *nocc, int nslices,
                           double *const *K_dev, void *stream);
/* FP64 Coulomb build of every molecule (Eqs. df-j-1/2), graph-captured likewise;
 * rho goes to each context's internal buffer. */
df_status df_batch_build_J(df_batch *b, const double *const *D_dev, double *const *J_dev, void *stream);
/* Autotuner: times, on this batch, every combination of the first GEMM's
 * tile (CTA-pair 256 x 128 tiles with the (P, mu) rows on the MMA's M side,
 * possible when every molecule's orbitals fit one 128-row tile, or
 * single-CTA 128 x 128 tiles with the orbitals on M), the K-split cap of the
 * second GEMM (1, 2, 4 or 8, at most the context's own split) and the
 * molecule order of the unit lists (as given, or most expensive first), and
 * keeps the fastest.  choice (host, 3 ints, may be NULL): [0] K-split cap,
 * [1] order, [2] first-GEMM tile (1 pair, 0 single).  Synchronises
 * `stream`. */
df_status df_batch_autotune(df_batch *b, const double *const *C_dev, const int *nocc, int nslices,
                            double *const *K_dev, void *stream, int *choice);

/* ---- Learned slice-count predictor (per 128-function auxiliary block) ----
 * A 16 -> 64 -> 64 -> 8 MLP (FP32, ReLU, softmax over slice counts 1..8)
 * with hand-written CUDA forward, backward and Adam kernels.  Parameters are
 * one float buffer of df_mlp_num_params() values: W1[64][16], b1[64],
 * W2[64][64], b2[64], W3[8][64], b3[8] (y = W x + b).  The paper has no such
 * part; it extends its closing suggestion (Section 5) of tying the emulation
 * level to the change of the density matrix. */
typedef struct df_mlp df_mlp;
df_status df_mlp_create(df_mlp **out);  /* parameters zero; set them with df_mlp_set_params */
void df_mlp_destroy(df_mlp *m);
int df_mlp_num_params(void);
df_status df_mlp_set_params(df_mlp *m, const float *host, int n);  /* also resets the Adam moments */
df_status df_mlp_get_params(const df_mlp *m, float *host, int n);
/* probs_dev [n][8] = softmax(MLP(X_dev [n][16])). */
df_status df_mlp_forward(df_mlp *m, const float *X_dev, int n, float *probs_dev, void *stream);
/* Gradient of the mean cross-entropy over (X_dev, y_dev in 0..7) into
 * grad_host (df_mlp_num_params floats) and the loss into loss_host (either
 * may be NULL; non-NULL synchronises). */
df_status df_mlp_gradients(df_mlp *m, const float *X_dev, const int *y_dev, int n, float *grad_host,
                           float *loss_host, void *stream);
/* One Adam step (beta 0.9/0.999) on the mean cross-entropy. */
df_status df_mlp_train_step(df_mlp *m, const float *X_dev, const int *y_dev, int n, float lr, float *loss_host,
                            void *stream);
/* 16 features per auxiliary block into F_dev [nblk][16]: block max and
 * Frobenius norm of B, mean and spread of its row exponents, relative
 * weight, small-row fraction (computed once from B), plus the iteration's
 * log10 tolerance tau, ||D_k - D_{k-1}||_F, Delta E_rel and the rule's slice
 * count. */
df_status df_block_features(df_ctx *ctx, int nocc, double tau, double dD, double dE, int s_rule, float *F_dev,
                            void *stream);
/* Attach the slice-count network to a context for df_build_K(nslices = -2)
 * (the context keeps the pointer; NULL detaches; the caller keeps the network
 * alive while attached).  At the current Table 1 level L (count s_L, printed
 * accuracy tau_L) each build computes the 16 block features
 * (df_block_features with tau_L, the density change measured by the last two
 * df_build_J calls, the last relative energy change seen by
 * df_adaptive_next, and s_L), runs the network, and takes for block b the
 * most probable count s_b, or s_L when that probability is below min_conf
 * (in (0, 1]); a count above s_L only pays for another block below s_L, so
 * when no block is below s_L every block takes s_L.  After the first GEMM
 * and the X split it checks, without any
 * FP64 reference, the a-priori error bound of every block's K_b
 *   beta_b(s) = kb_b 1.01 (s + 1) 2^(-8 s) (2^(2 E_b) + 2 nao 2^(F_b + E_c + E_b))
 *               + kb_b 2^(2 E_b - 52)
 * (kb_b = functions in the block x nocc, the contraction length; E_b the
 * largest exponent of the block's X rows, F_b of its B rows, E_c of C's
 * columns; the first term bounds the slice truncation of both GEMMs, the
 * second the FP64 roundings): the counts pass if
 * sum_b beta_b(s_b) <= (1 + 1e-12) sum_b beta_b(s_L), i.e. the learned
 * build's bound is at most the rule's (the 1e-12 absorbs the rounding of the
 * sums; a block whose bound is that far below the others may keep any count).  Otherwise the blocks with s_b < s_L are raised to s_L,
 * largest beta_b(s_b) first, until it holds, and the first GEMM and the X
 * split are run again with the raised counts. */
df_status df_set_predictor(df_ctx *ctx, df_mlp *net, float min_conf);

/* Labels: err_host [nblk][8] = max |K_b(s) - K_b(FP64)| of every block at
 * s = 1..8 (the emulated build against cuBLAS FP64, per block), *kmax_host =
 * max|K(FP64)|.  Runs s_max + 1 builds; synchronises. */
df_status df_block_errors(df_ctx *ctx, const double *C_dev, int nocc, double *err_host, double *kmax_host,
                          void *stream);

/* Phases timed when profiling is on (CUDA events on the call's stream). */
#define DF_PHASE_SPLIT_C 0  /* C -> digit planes */
#define DF_PHASE_GEMM1 1    /* X = B C on the tensor cores (or cuBLAS DGEMM in FP64 mode) */
#define DF_PHASE_SPLIT_X 2  /* X -> per-(block, mu) digit planes */
#define DF_PHASE_GEMM2 3    /* K_b = X_b X_b^T on the tensor cores (or cuBLAS DSYRK) */
#define DF_PHASE_REDUCE 4   /* K = sum_b K_b */
#define DF_PHASE_RHO 5      /* rho = B . D */
#define DF_PHASE_COULOMB 6  /* J = B^T rho */
#define DF_PHASE_ENERGY 7   /* energy reductions */
#define DF_NPHASES 8

/* Turn per-phase event timing on or off (off by default; costs two event
 * records per phase). */
df_status df_set_profiling(df_ctx *ctx, int on);
/* Summed phase times (ms) and record counts since the last read, for the
 * DF_NPHASES phases; waits for the recorded events and clears them. */
df_status df_phase_times(df_ctx *ctx, double *ms, int *count);

/* Device bytes held by the context's workspaces. */
int64_t df_workspace_bytes(const df_ctx *ctx);

/* Block sparsity found by df_setup (the Schwarz screening of Section 2.1
 * zeroes a screened AO pair (mu, nu) in every B_P; the paper's FLOP model
 * counts the surviving pairs as N_scr).  At setup the library records, per mu,
 * which 64-wide chunks of nu hold a nonzero B_P mu nu for some P; when some
 * chunk is zero (and nao <= 2048) the first exchange GEMM runs only the
 * nonzero 64-wide K tiles of each 128-row tile of B's (P, mu) rows, and rho
 * and J skip the zero chunks.  Skipped terms are exact zeros: every result is
 * the one of the dense build.  frac_ktiles: nonzero K tiles / all of the first
 * GEMM's row tiles; frac_chunks: nonzero (mu, chunk) pairs of the upper
 * triangle / all.  Both 1 for a B without zero chunks.  DF_ERR_STATE before
 * setup. */
df_status df_sparsity(const df_ctx *ctx, double *frac_ktiles, double *frac_chunks);

/* Execution options of a context (they change speed, never results: every
 * option gives bit-identical K).
 *
 * DF_OPT_CLUSTER_PAIRS — whether the two slice GEMMs of df_build_K /
 * df_build_K_blocks (Section 3.2's slice products) run on CTA pairs: a
 * cluster of two CTAs whose M = 256 tcgen05 MMA (cta_group::2) covers two
 * output tiles that share the stacked B operand, each CTA staging its own A
 * tile and half of B.  0 never; 1 (default) the first GEMM whenever its
 * occupied-orbital tiles pair up (every pair is useful there); 2 both GEMMs
 * wherever the layout pairs (the second GEMM's pairs also compute one lower
 * tile per pair of AO tile rows, which on GB300 costs more than pairing
 * saves).
 *
 * Returns DF_ERR_ARG for an unknown option or value; the context is unchanged. */
#define DF_OPT_CLUSTER_PAIRS 1
/* DF_OPT_SPARSE — whether the builds use the block sparsity of a screened B
 * (df_sparsity): 1 (default) when df_setup found zero chunks, 0 never. */
#define DF_OPT_SPARSE 2
/* DF_OPT_JK_OVERLAP — CTAs per SM of the rho and J kernels that df_build_JK
 * runs beside the X split: 1..4 (default 4, the fastest at 240 atoms), 0 = no
 * overlap (J, then K, in the caller's stream). */
#define DF_OPT_JK_OVERLAP 3
df_status df_set_option(df_ctx *ctx, int option, int value);

#ifdef __cplusplus
}
#endif
#endif /* DF_H_ */
