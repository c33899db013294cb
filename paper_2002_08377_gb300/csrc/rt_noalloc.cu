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
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current); make that first call
// before any stream capture.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "rt_internal.cuh"

namespace {

constexpr int kMaxBlocks = 2048;           // partial sums the array holds
constexpr int kMaxCellsPerBlock = 4096;    // cells one block may sum
constexpr int64_t kMaxCells = (int64_t)kMaxBlocks * kMaxCellsPerBlock;
constexpr int kThreads = 256;
constexpr int kParts = 12;                 // partial sums per block
constexpr int kMaxDevices = 64;

// [kMaxBlocks][kParts] block partial sums, then the 16 results
static __device__ __align__(256) double g_totals_scratch[kMaxBlocks * kParts + 16];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_totals_scratch on `dev` (which must be current).
cudaError_t scratch_on(int dev, double **ptr) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    double *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_totals_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Block b sums cells [b cpb, min(n, (b + 1) cpb)) in a fixed order: warp w
// takes every eighth cell, lanes split the angles, warps combine in order.
template <typename R>
__global__ void totals_blocks_kernel(const R *__restrict__ I, const double *__restrict__ dir,
                                     const double *__restrict__ wt,
                                     const double *__restrict__ vol,
                                     const rt::GasDyn *__restrict__ gd,
                                     const double *__restrict__ ext, int64_t n, int A,
                                     int stride, int64_t cpb,
                                     double c_over_cbar, double inv_cbar, double *partial) {
  __shared__ double acc[kThreads / 32][kParts];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  double t[kParts] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  const int64_t c1 = c0 + cpb < n ? c0 + cpb : n;
  const double fp = 4.0 * rt::kPi;
  for (int64_t row = c0 + warp; row < c1; row += kThreads / 32) {
    const R *Ir = I + (size_t)row * stride;
    double e = 0, fx = 0, fy = 0, fz = 0;
    for (int a = lane; a < A; a += 32) {
      const double wi = wt[a] * (double)Ir[a];
      e += wi;
      fx += wi * dir[3 * a];
      fy += wi * dir[3 * a + 1];
      fz += wi * dir[3 * a + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      fx += __shfl_xor_sync(0xffffffffu, fx, o);
      fy += __shfl_xor_sync(0xffffffffu, fy, o);
      fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    if (lane == 0) {
      const double V = vol[row];
      const rt::GasDyn g = gd[row];
      t[0] += V * g.e;
      t[1] += V * c_over_cbar * fp * e;
      t[2] += V * ext[4 * row];
      t[3] += V * g.mx;
      t[4] += V * g.my;
      t[5] += V * g.mz;
      t[6] += V * fp * inv_cbar * fx;
      t[7] += V * fp * inv_cbar * fy;
      t[8] += V * fp * inv_cbar * fz;
      t[9] += V * ext[4 * row + 1];
      t[10] += V * ext[4 * row + 2];
      t[11] += V * ext[4 * row + 3];
    }
  }
  if (lane == 0)
    for (int k = 0; k < kParts; ++k) acc[warp][k] = t[k];
  __syncthreads();
  if (threadIdx.x < kParts) {
    double s = 0;
    for (int w = 0; w < kThreads / 32; ++w) s += acc[w][threadIdx.x];
    partial[(size_t)blockIdx.x * kParts + threadIdx.x] = s;
  }
}

// Component k summed over the blocks in block order; out16 as rt_totals.
__global__ void totals_combine_kernel(const double *__restrict__ partial, int nblocks,
                                      double *out16) {
  __shared__ double v[kParts];
  const int k = threadIdx.x;
  if (k < kParts) {
    double s = 0;
    for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * kParts + k];
    v[k] = s;
    out16[k] = s;
  }
  __syncthreads();
  if (k == 0) out16[12] = v[0] + v[1] + v[2];
  if (k < 3) out16[13 + k] = v[3 + k] + v[6 + k] + v[9 + k];
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
  int64_t cpb = (s->n_cells + kMaxBlocks - 1) / kMaxBlocks;
  if (cpb < 64) cpb = 64;
  const int nb = (int)((s->n_cells + cpb - 1) / cpb);
  const double coc = s->params.c / s->params.cbar, icb = 1.0 / s->params.cbar;
  const void *I = s->d_I[s->cur];
  if (s->precision == RT_FP32)
    totals_blocks_kernel<float><<<nb, kThreads, 0, s->stream>>>(
        (const float *)I, s->d_dir64, s->d_wt64, s->d_volume, s->d_gd, s->d_ext, s->n_cells,
        s->n_angles, s->row_stride, cpb, coc, icb, partial);
  else
    totals_blocks_kernel<double><<<nb, kThreads, 0, s->stream>>>(
        (const double *)I, s->d_dir64, s->d_wt64, s->d_volume, s->d_gd, s->d_ext, s->n_cells,
        s->n_angles, s->row_stride, cpb, coc, icb, partial);
  totals_combine_kernel<<<1, 32, 0, s->stream>>>(partial, nb, res);
  s->launches += 2;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, 16 * sizeof(double), cudaMemcpyDeviceToHost,
                                            s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return fail(s, RT_ERR_CUDA, cudaGetErrorString(e));
  return RT_OK;
}
