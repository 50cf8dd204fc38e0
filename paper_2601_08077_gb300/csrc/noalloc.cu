// df_emulated_gemm_static: the FP64-emulated product of df_emulated_gemm,
// computed without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a framework whose caching
// allocator or fixed arena has already reserved nearly all device memory (a
// library-side cudaMalloc then fails, or fragments the arena), or a latency-
// sensitive loop that cannot afford the device-wide synchronisation that
// cudaMalloc and cudaFree imply.  This entry point takes its scratch (digit
// planes, exponents, the status word) from one file-scope __device__ array
// of kStaticScratchBytes instead.  The caller still passes the inputs and the
// output.
//
// The array lives on every GPU that loads this library until the process
// exits.  Its device address is looked up once per device, with that device
// current, on the first call made on that device.  That first call should
// therefore come before any stream capture.  The address is kept for the
// life of the process: after cudaDeviceReset the cached address no longer
// belongs to the device's new context, so a process that resets a device
// must not call this entry point on that device again.  All calls share the array and it
// keeps the contents of the last call; the status word is cleared at the start
// of each call and every other byte that is read is written first.  Calls
// whose GPU work overlaps (for example from two host threads on two streams)
// race on the array.
#include "df_internal.h"

#include <cstring>
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_dev[kMaxDevices] = {nullptr};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (set up once per device).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_dev[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = ptr;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" df_status df_emulated_gemm_static(const double *A, const double *B, int M, int N, int K, int nslices,
                                             double *out, void *stream) {
  if (!A || !B || !out || M <= 0 || N <= 0 || K <= 0 || nslices < 1 || nslices > DF_S_MAX) return DF_ERR_ARG;
  const long long ld = ((long long)K + 7) / 8 * 8;
  // A B^T with B == A (a Gram matrix): one split serves both sides, as in
  // df_emulated_gemm, so only one operand's planes and exponents are carved
  const bool same = A == B && M == N;
  // carve the scratch: status word, exponents of A (and B), digit planes of A (and B)
  const size_t off_status = 0;
  const size_t off_ea = align256(off_status + sizeof(int));
  const size_t off_eb = align256(off_ea + sizeof(int) * (size_t)M);
  const size_t off_ad = same ? off_eb : align256(off_eb + sizeof(int) * (size_t)N);
  const size_t off_bd = align256(off_ad + sizeof(uint16_t) * (size_t)nslices * M * ld);
  const size_t need = same ? off_bd : align256(off_bd + sizeof(uint16_t) * (size_t)nslices * N * ld);
  if (need > kStaticScratchBytes) return DF_ERR_SCRATCH;

  void *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return DF_ERR_CUDA;
  unsigned char *s = static_cast<unsigned char *>(base);
  int *status = reinterpret_cast<int *>(s + off_status);
  int *ea = reinterpret_cast<int *>(s + off_ea);
  uint16_t *Ad = reinterpret_cast<uint16_t *>(s + off_ad);
  int *eb = same ? ea : reinterpret_cast<int *>(s + off_eb);
  uint16_t *Bd = same ? Ad : reinterpret_cast<uint16_t *>(s + off_bd);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = df::launch_split_rows_bf16(A, M, K, K, nslices, ea, Ad, ld, (long long)M * ld, st);
  if (e == cudaSuccess && !same)
    e = df::launch_split_rows_bf16(B, N, K, K, nslices, eb, Bd, ld, (long long)N * ld, st);
  if (e != cudaSuccess) return DF_ERR_CUDA;
  CUtensorMap ta, tb;
  if (!df::make_tmap_bf16(&ta, Ad, K, M, nslices, ld, (long long)M * ld) ||
      !df::make_tmap_bf16(&tb, Bd, K, N, nslices, ld, (long long)N * ld))
    return DF_ERR_CUDA;
  df::SgParams p;
  std::memset(&p, 0, sizeof(p));
  p.layout = df::kLayoutGrid;
  p.mode = df::kModeGemm;
  p.nt_m = (M + df::kTile - 1) / df::kTile;
  p.nt_n = (N + df::kTile - 1) / df::kTile;
  p.nunits = p.nt_m * p.nt_n;
  p.m_valid = M;
  p.n_valid = N;
  p.ktiles = (K + df::kKTile - 1) / df::kKTile;
  p.s_fixed = nslices;
  for (int q = 0; q <= 8; ++q) p.shiftT[q] = df::fixed_point_shift(q, (long long)p.ktiles * df::kKTile);
  p.ea = ea;
  p.eb = eb;
  p.out = out;
  p.out_ld = N;
  p.status = status;
  e = df::launch_slice_gemm(p, ta, tb, st);
  if (e != cudaSuccess) return DF_ERR_CUDA;
  int h = 0;
  e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return DF_ERR_CUDA;
  return h ? DF_ERR_TIMEOUT : DF_OK;
}
