// Batched J/K builds over many molecules of uneven size.
//
// One exchange build for n molecules is
//   per molecule   split C                       (HBM, small)
//   ONE launch     first exchange GEMM over the work units of all molecules
//                  (persistent, grouped: a unit finds its molecule by a
//                  prefix table, whose parameters and TMA maps live in
//                  device memory)
//   per molecule   split X
//   ONE launch     second exchange GEMM over all molecules' units
//   per molecule   reduce K
// and the whole sequence is captured once as a CUDA graph and replayed.  The
// autotuner times the K-split depth of the second GEMM and the order of the
// molecules in the unit list (as given, or most expensive first) on the
// actual batch and keeps the fastest.
#include "df_ctx.h"

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

struct df_batch {
  std::vector<df_ctx *> ctx;
  int nsplit_cap = 8;
  int order = 1;  // 0: as given, 1: most expensive first
  int tile1 = 1;  // first GEMM: 1 CTA-pair 256 x 128 tiles when possible, 0 single-CTA 128 x 128
  bool graphs = true;
  // grouped-launch tables (device)
  df::SgParams *params1 = nullptr, *params2 = nullptr;
  CUtensorMap *maps1 = nullptr, *maps2 = nullptr;
  int *off1 = nullptr, *off2 = nullptr;
  int total1 = 0, total2 = 0;
  int *status = nullptr;
  std::vector<int> nsplit;  // per molecule, in molecule order
  std::vector<int> nocc;
  int tables_for_s = -1;
  bool pairs1 = false;  // first GEMM on CTA pairs (swapped layout, tables in tile pairs)
  // side streams for the per-molecule kernels (X split, reduce, rho and J):
  // molecule i runs on side[i % kFan] between a fork and a join of the
  // caller's stream, in eager launches and inside a captured graph alike
  static constexpr int kFan = 4;
  cudaStream_t side[kFan] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kFan] = {};
  // graph cache
  cudaGraphExec_t exec_K = nullptr, exec_J = nullptr;
  std::vector<const void *> key_K, key_J;
  int key_s = -1;
};

namespace {

df_status cerr(cudaError_t e) { return e == cudaSuccess ? DF_OK : DF_ERR_CUDA; }

void drop_graph(cudaGraphExec_t &g) {
  if (g) cudaGraphExecDestroy(g);
  g = nullptr;
}

// The side streams start after everything enqueued on st so far.
cudaError_t fork(df_batch *b, cudaStream_t st) {
  cudaError_t e = cudaEventRecord(b->ev_fork, st);
  for (int k = 0; k < df_batch::kFan && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->ev_fork, 0);
  return e;
}

// st continues after everything enqueued on the side streams so far.
cudaError_t join(df_batch *b, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < df_batch::kFan && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->ev_join[k], b->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_join[k], 0);
  }
  return e;
}

// Molecule order for the unit lists.
std::vector<int> unit_order(const df_batch *b, const int *nocc) {
  std::vector<int> ord(b->ctx.size());
  std::iota(ord.begin(), ord.end(), 0);
  if (b->order == 1) {
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      const df_ctx *a = b->ctx[x], *c = b->ctx[y];
      const double ca = (double)a->naux * a->nao * a->nao * nocc[x];
      const double cc = (double)c->naux * c->nao * c->nao * nocc[y];
      return ca > cc;
    });
  }
  return ord;
}

df_status build_tables(df_batch *b, const int *nocc) {
  const int n = (int)b->ctx.size();
  std::vector<df::SgParams> p1(n), p2(n);
  std::vector<CUtensorMap> m1(2 * n), m2(2 * n);
  std::vector<int> o1(n + 1, 0), o2(n + 1, 0);
  const std::vector<int> ord = unit_order(b, nocc);
  b->nsplit.assign(n, 1);
  // the first GEMM runs on CTA pairs when every molecule's orbitals fit one tile
  // (the swapped layout; one slice count per molecule, so pairs may cross blocks)
  b->pairs1 = b->tile1 == 1;
  for (int i = 0; i < n; ++i) b->pairs1 = b->pairs1 && b->ctx[i]->pair_mode >= 1 && nocc[i] <= df::kTile;
  for (int k = 0; k < n; ++k) {
    const int i = ord[k];
    df_ctx *c = b->ctx[i];
    const int ns = std::max(1, std::min(b->nsplit_cap, c->nsplit));
    b->nsplit[i] = ns;
    if (!df::gemm1_setup(c, nocc[i], p1[k], m1[2 * k], m1[2 * k + 1], b->pairs1 ? 2 : 0)) return DF_ERR_CUDA;
    if (!df::gemm2_setup(c, nocc[i], ns, p2[k], m2[2 * k])) return DF_ERR_CUDA;
    m2[2 * k + 1] = m2[2 * k];
    if (b->pairs1) p1[k].npairs = (int)df::slice_gemm_pairs(p1[k]);
    o1[k + 1] = o1[k] + (b->pairs1 ? p1[k].npairs : p1[k].nunits);
    o2[k + 1] = o2[k] + p2[k].nunits;
  }
  b->total1 = o1[n];
  b->total2 = o2[n];
  cudaError_t e = cudaMemcpy(b->params1, p1.data(), sizeof(df::SgParams) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->params2, p2.data(), sizeof(df::SgParams) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->maps1, m1.data(), sizeof(CUtensorMap) * 2 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->maps2, m2.data(), sizeof(CUtensorMap) * 2 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->off1, o1.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->off2, o2.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
  b->nocc.assign(nocc, nocc + n);
  return cerr(e);
}

// Every launch of one batched exchange build (no host synchronisation: capturable).
df_status enqueue_K(df_batch *b, const double *const *C, const int *nocc, int s, double *const *K,
                    cudaStream_t st) {
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; ++i) {
    df_ctx *c = b->ctx[i];
    const long long c_plane = (long long)c->nocc_max * c->ld_nao;
    if (df::launch_split_cols_bf16(C[i], c->nao, nocc[i], s, c->eC, c->Cd, c->ld_nao, c_plane, st) != cudaSuccess)
      return DF_ERR_CUDA;
  }
  for (int i = 0; i < n; ++i)
    if (cudaMemsetAsync(b->ctx[i]->rowE, 0x80, sizeof(int) * (size_t)b->ctx[i]->nblk * b->ctx[i]->nao, st) !=
        cudaSuccess)
      return DF_ERR_CUDA;
  df::SgGroup g1{b->params1, b->maps1, b->off1, n, b->total1};
  if (df::launch_slice_gemm_grouped(b->pairs1 ? df::kModeXs : df::kModeX, g1, b->status, 0, st, b->pairs1) !=
      cudaSuccess)
    return DF_ERR_CUDA;
  if (fork(b, st) != cudaSuccess) return DF_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    df_ctx *c = b->ctx[i];
    df::ShiftTable t1;
    const long long k1 = (long long)((c->nao + df::kKTile - 1) / df::kKTile) * df::kKTile;
    for (int q = 0; q <= 8; ++q) t1.v[q] = df::fixed_point_shift(q, k1);
    if (df::launch_split_xblocks(reinterpret_cast<const long long *>(c->X), c->naux, c->nao, nocc[i], s, c->eB,
                                 c->eC, c->sblk, t1, c->rowE, c->eX, c->Xd, df::xdigit_ld(nocc[i]), c->nblk,
                                 b->side[i % df_batch::kFan]) != cudaSuccess)
      return DF_ERR_CUDA;
  }
  if (join(b, st) != cudaSuccess) return DF_ERR_CUDA;
  df::SgGroup g2{b->params2, b->maps2, b->off2, n, b->total2};
  if (df::launch_slice_gemm_grouped(df::kModeKPart, g2, b->status, 0, st) != cudaSuccess) return DF_ERR_CUDA;
  if (fork(b, st) != cudaSuccess) return DF_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    df_ctx *c = b->ctx[i];
    df::ShiftTable tt;
    const long long kb = df::xdigit_ld(nocc[i]);
    for (int q = 0; q <= 8; ++q) tt.v[q] = df::fixed_point_shift(q, kb);
    if (df::launch_kpart_reduce(c->Rp, c->eX, c->sblk, tt, c->nao, c->nblk, b->nsplit[i], K[i],
                                b->side[i % df_batch::kFan]) != cudaSuccess)
      return DF_ERR_CUDA;
  }
  return join(b, st) == cudaSuccess ? DF_OK : DF_ERR_CUDA;
}

df_status prepare(df_batch *b, const int *nocc, int s, cudaStream_t st) {
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; ++i) {
    df_ctx *c = b->ctx[i];
    if (!c->ready || nocc[i] <= 0 || nocc[i] > c->nocc_max || s < 1 || s > c->s_max) return DF_ERR_ARG;
    std::vector<int> sb(c->nblk, s);
    df_status r = df::ctx_upload_slices(c, sb.data(), st);
    if (r != DF_OK) return r;
  }
  bool same = b->tables_for_s == s && (int)b->nocc.size() == n;
  for (int i = 0; same && i < n; ++i) same = b->nocc[i] == nocc[i];
  if (!same) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return DF_ERR_CUDA;
    df_status r = build_tables(b, nocc);
    if (r != DF_OK) return r;
    b->tables_for_s = s;
    drop_graph(b->exec_K);
  }
  return DF_OK;
}

}  // namespace

extern "C" {

df_status df_batch_create(df_batch **out, df_ctx *const *ctxs, int n) {
  if (!out || !ctxs || n <= 0) return DF_ERR_ARG;
  *out = nullptr;
  df_batch *b = new (std::nothrow) df_batch();
  if (!b) return DF_ERR_OOM;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) {
      delete b;
      return DF_ERR_ARG;
    }
    // each molecule needs its own context: their kernels run concurrently
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) {
        delete b;
        return DF_ERR_ARG;
      }
  }
  b->ctx.assign(ctxs, ctxs + n);
  cudaError_t e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int k = 0; k < df_batch::kFan && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->params1, sizeof(df::SgParams) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->params2, sizeof(df::SgParams) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->maps1, sizeof(CUtensorMap) * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->maps2, sizeof(CUtensorMap) * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->off1, sizeof(int) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->off2, sizeof(int) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int));
  if (e != cudaSuccess) {
    df_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? DF_ERR_OOM : DF_ERR_CUDA;
  }
  *out = b;
  return DF_OK;
}

void df_batch_destroy(df_batch *b) {
  if (!b) return;
  drop_graph(b->exec_K);
  drop_graph(b->exec_J);
  for (int k = 0; k < df_batch::kFan; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  cudaFree(b->params1);
  cudaFree(b->params2);
  cudaFree(b->maps1);
  cudaFree(b->maps2);
  cudaFree(b->off1);
  cudaFree(b->off2);
  cudaFree(b->status);
  delete b;
}

df_status df_batch_set_graphs(df_batch *b, int on) {
  if (!b) return DF_ERR_ARG;
  b->graphs = on != 0;
  return DF_OK;
}

df_status df_batch_build_K(df_batch *b, const double *const *C, const int *nocc, int nslices, double *const *K,
                           void *stream) {
  if (!b || !C || !nocc || !K) return DF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  df_status r = prepare(b, nocc, nslices, st);
  if (r != DF_OK) return r;
  const int n = (int)b->ctx.size();
  if (!b->graphs || st == nullptr) return enqueue_K(b, C, nocc, nslices, K, st);
  std::vector<const void *> key;
  for (int i = 0; i < n; ++i) {
    key.push_back(C[i]);
    key.push_back(K[i]);
  }
  if (!b->exec_K || key != b->key_K || b->key_s != nslices) {
    drop_graph(b->exec_K);
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DF_ERR_CUDA;
    df_status er = enqueue_K(b, C, nocc, nslices, K, st);
    cudaError_t ee = cudaStreamEndCapture(st, &graph);
    if (er != DF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return er;
    }
    if (ee != cudaSuccess) return DF_ERR_CUDA;
    ee = cudaGraphInstantiate(&b->exec_K, graph, 0);
    cudaGraphDestroy(graph);
    if (ee != cudaSuccess) return DF_ERR_CUDA;
    b->key_K = key;
    b->key_s = nslices;
  }
  return cerr(cudaGraphLaunch(b->exec_K, st));
}

df_status df_batch_build_J(df_batch *b, const double *const *D, double *const *J, void *stream) {
  if (!b || !D || !J) return DF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; ++i)
    if (!b->ctx[i]->ready) return DF_ERR_STATE;
  auto enqueue = [&]() -> df_status {
    if (fork(b, st) != cudaSuccess) return DF_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
      df_ctx *c = b->ctx[i];
      cudaStream_t si = b->side[i % df_batch::kFan];
      const uint32_t *mk = df::use_mask_mu(c);
      if (df::launch_rho(c->B, D[i], c->naux, c->nao, c->rho, si, mk, c->packed, nullptr, 0, c->sparse) != cudaSuccess) return DF_ERR_CUDA;
      if (df::launch_coulomb(c->B, c->rho, c->naux, c->nao, J[i], si, mk, c->packed) != cudaSuccess)
        return DF_ERR_CUDA;
    }
    return join(b, st) == cudaSuccess ? DF_OK : DF_ERR_CUDA;
  };
  if (!b->graphs || st == nullptr) return enqueue();
  std::vector<const void *> key;
  for (int i = 0; i < n; ++i) {
    key.push_back(D[i]);
    key.push_back(J[i]);
  }
  if (!b->exec_J || key != b->key_J) {
    drop_graph(b->exec_J);
    // the Coulomb kernel sets its shared-memory attribute on first use: do it outside capture
    for (int i = 0; i < n; ++i)
      if (df::launch_coulomb(b->ctx[i]->B, b->ctx[i]->rho, b->ctx[i]->naux, b->ctx[i]->nao, J[i], st, nullptr,
                             b->ctx[i]->packed) !=
          cudaSuccess)
        return DF_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DF_ERR_CUDA;
    df_status er = enqueue();
    cudaError_t ee = cudaStreamEndCapture(st, &graph);
    if (er != DF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return er;
    }
    if (ee != cudaSuccess) return DF_ERR_CUDA;
    ee = cudaGraphInstantiate(&b->exec_J, graph, 0);
    cudaGraphDestroy(graph);
    if (ee != cudaSuccess) return DF_ERR_CUDA;
    b->key_J = key;
  }
  return cerr(cudaGraphLaunch(b->exec_J, st));
}

df_status df_batch_autotune(df_batch *b, const double *const *C, const int *nocc, int nslices, double *const *K,
                            void *stream, int *choice) {
  if (!b || !C || !nocc || !K) return DF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool graphs = b->graphs;
  b->graphs = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // the first GEMM's CTA-pair tiles exist only when every molecule's orbitals fit one tile
  bool pairs_possible = true;
  for (size_t i = 0; i < b->ctx.size(); ++i)
    pairs_possible = pairs_possible && b->ctx[i]->pair_mode >= 1 && nocc[i] <= df::kTile;
  float best = 1e30f;
  int best_ns = b->nsplit_cap, best_ord = b->order, best_tile = pairs_possible ? 1 : 0;
  df_status r = DF_OK;
  const int caps[4] = {1, 2, 4, 8};
  for (int tile = pairs_possible ? 1 : 0; tile >= 0 && r == DF_OK; --tile) {
    for (int ord = 0; ord < 2 && r == DF_OK; ++ord) {
      for (int ci = 0; ci < 4 && r == DF_OK; ++ci) {
        b->tile1 = tile;
        b->order = ord;
        b->nsplit_cap = caps[ci];
        b->tables_for_s = -1;
        r = df_batch_build_K(b, C, nocc, nslices, K, stream);  // warm-up (and tables)
        if (r != DF_OK) break;
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 2 && r == DF_OK; ++rep) r = df_batch_build_K(b, C, nocc, nslices, K, stream);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) r = DF_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == DF_OK && ms < best) {
          best = ms;
          best_ns = caps[ci];
          best_ord = ord;
          best_tile = tile;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->nsplit_cap = best_ns;
  b->order = best_ord;
  b->tile1 = best_tile;
  b->tables_for_s = -1;
  b->graphs = graphs;
  drop_graph(b->exec_K);
  if (choice) {
    choice[0] = best_ns;
    choice[1] = best_ord;
    choice[2] = best_tile;
  }
  return r;
}

}  // extern "C"
