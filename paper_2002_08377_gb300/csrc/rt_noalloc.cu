// Conserved totals for callers that cannot allocate device memory.
//
// rt_totals keeps its per-block partial sums in a buffer that rt_create
// allocated.  rt_totals_noalloc computes the same sixteen numbers but keeps
// the partial sums and the result in one file-scope device array, so a call
// needs no allocation of any kind: it suits callers that run where
// cudaMalloc is off limits -- a thread that must not block on the driver's
// allocator, code whose device memory is entirely owned by another
// allocator (a framework's caching pool), or a program that sizes all of its
// device memory once at start-up.
//
// Limits and sharing:
//   - at most kMaxBlocks x kMaxCellsPerBlock = 8,388,608 cells; larger states
//     are rejected with RT_ERR_ARG;
//   - the array (197 KB) exists once on every device that loads the library
//     and stays there until the process exits;
//   - every call on a device reuses the same array, so calls whose GPU work
//     overlaps (different streams, or different states on one device) race
//     and must be serialised by the caller;
//   - each call writes every partial it later reads, so nothing has to be
//     cleared between calls.
// The first call in a context looks up the array's device address with
// cudaGetSymbolAddress (with that device current); make that first call
// before any stream capture.  The address is kept per device together with
// the identifier of the context it was looked up in, and looked up again
// when the current context differs (after cudaDeviceReset, say).
// The sums are those of rt_totals, computed by the same kernels: blocks of
// 64 cells as rt_totals sums them while the state has at most 2048 x 64 =
// 131,072 cells (bit-identical results), larger blocks beyond that (the
// same totals to rounding, not bit for bit).
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "rt_internal.cuh"

namespace {

constexpr int kMaxBlocks = 2048;           // partial sums the array holds
constexpr int kMaxCellsPerBlock = 4096;    // cells one block may sum
constexpr int64_t kMaxCells = (int64_t)kMaxBlocks * kMaxCellsPerBlock;
constexpr int kParts = 12;                 // partial sums per block
constexpr int kMaxDevices = 64;

// [kMaxBlocks][kParts] block partial sums, then the 16 results
static __device__ __align__(256) double g_totals_scratch[kMaxBlocks * kParts + 16];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};

// Device address of g_totals_scratch on `dev` (which must be current), kept
// for the context it was looked up in.
cudaError_t scratch_on(int dev, double **ptr) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long ctx = rt::current_context_id();
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    double *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_totals_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *ptr = g_scratch_ptr[dev];
  return cudaSuccess;
}

int fail(rt_state *s, int code, const char *msg) {
  s->err = msg;
  return code;
}

}  // namespace

extern "C" int rt_totals_noalloc(rt_state *s, double out[16]) {
  if (!s) return RT_ERR_ARG;
  if (!out) return fail(s, RT_ERR_ARG, "rt_totals_noalloc: out is NULL");
  if (s->n_cells > kMaxCells) {
    char buf[160];
    snprintf(buf, sizeof buf,
             "rt_totals_noalloc handles at most %lld cells; this state has %lld (use rt_totals)",
             (long long)kMaxCells, (long long)s->n_cells);
    return fail(s, RT_ERR_ARG, buf);
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(s, RT_ERR_CUDA, cudaGetErrorString(e));
  if (dev != s->device)
    return fail(s, RT_ERR_STATE, "rt_totals_noalloc: the state's device is not the current device");
  double *scratch = nullptr;
  e = scratch_on(dev, &scratch);
  if (e != cudaSuccess) return fail(s, RT_ERR_CUDA, cudaGetErrorString(e));
  double *partial = scratch, *res = scratch + (size_t)kMaxBlocks * kParts;
  // rt_totals' blocks while they fit the array, else fewer, larger blocks
  int64_t cpb = (s->n_cells + kMaxBlocks - 1) / kMaxBlocks;
  if (cpb < rt::totals_block_cells) cpb = rt::totals_block_cells;
  e = rt::launch_totals_with(s, partial, cpb, res);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, 16 * sizeof(double), cudaMemcpyDeviceToHost,
                                            s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return fail(s, RT_ERR_CUDA, cudaGetErrorString(e));
  return RT_OK;
}
