// Auxiliary kernels: caller<->internal cell order, the upwind positivity
// bound, lab-frame moments (Sec. 2.1), conserved totals (Sec. 2.3.1) and the
// gas read-back.  None of these is on the per-step hot path.
#include <cuda_runtime.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int kThreads = 256;

// dst[ic][q] = src[cell_of[ic]][angle_of[q]]  (caller order -> internal order;
// internal rows `stride` reals apart).  A warp keeps its lanes' entries of
// the angle map in registers (A <= 128) and moves two rows per iteration of
// a grid-stride loop, so that each warp has two rows' loads in flight.
constexpr int kMapPerLane = 4;  // 128 angles / 32 lanes
template <typename R>
__global__ void permute_in_kernel(const R *__restrict__ src, R *__restrict__ dst,
                                  const int64_t *__restrict__ cell_of,
                                  const int32_t *__restrict__ angle_of, int64_t n, int A,
                                  int stride) {
  const int lane = threadIdx.x % 32;
  int ang[kMapPerLane];
#pragma unroll
  for (int j = 0; j < kMapPerLane; ++j) ang[j] = lane + 32 * j < A ? angle_of[lane + 32 * j] : 0;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; row < n;
       row += 2 * nw) {
    const int64_t r2 = row + nw < n ? row + nw : row;
    const R *s1 = src + (size_t)cell_of[row] * A, *s2 = src + (size_t)cell_of[r2] * A;
    R v1[kMapPerLane], v2[kMapPerLane];
#pragma unroll
    for (int j = 0; j < kMapPerLane; ++j)
      if (lane + 32 * j < A) {
        v1[j] = s1[ang[j]];
        v2[j] = s2[ang[j]];
      }
#pragma unroll
    for (int j = 0; j < kMapPerLane; ++j)
      if (lane + 32 * j < A) {
        dst[(size_t)row * stride + lane + 32 * j] = v1[j];
        dst[(size_t)r2 * stride + lane + 32 * j] = v2[j];  // r2 == row: the same value again
      }
  }
}

// dst[cell_of[ic]][angle_of[q]] = src[ic][q]  (internal order -> caller order)
template <typename R>
__global__ void permute_out_kernel(const R *__restrict__ src, R *__restrict__ dst,
                                   const int64_t *__restrict__ cell_of,
                                   const int32_t *__restrict__ angle_of, int64_t n, int A,
                                   int stride) {
  const int lane = threadIdx.x % 32;
  int ang[kMapPerLane];
#pragma unroll
  for (int j = 0; j < kMapPerLane; ++j) ang[j] = lane + 32 * j < A ? angle_of[lane + 32 * j] : 0;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; row < n;
       row += 2 * nw) {
    const int64_t r2 = row + nw < n ? row + nw : row;
    R v1[kMapPerLane], v2[kMapPerLane];
#pragma unroll
    for (int j = 0; j < kMapPerLane; ++j)
      if (lane + 32 * j < A) {
        v1[j] = src[(size_t)row * stride + lane + 32 * j];
        v2[j] = src[(size_t)r2 * stride + lane + 32 * j];
      }
    R *d1 = dst + (size_t)cell_of[row] * A, *d2 = dst + (size_t)cell_of[r2] * A;
#pragma unroll
    for (int j = 0; j < kMapPerLane; ++j)
      if (lane + 32 * j < A) {
        d1[ang[j]] = v1[j];
        d2[ang[j]] = v2[j];
      }
  }
}

// Host-memory forms: lane k takes caller column k of the row (contiguous on
// the host side) and the internal position pos_of[k].
template <typename R>
__global__ void permute_in_host_kernel(const R *__restrict__ src, R *__restrict__ dst,
                                       const int64_t *__restrict__ cell_of,
                                       const int32_t *__restrict__ pos_of, int64_t n, int A,
                                       int stride) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (row >= n) return;
  const R *s = src + (size_t)cell_of[row] * A;
  R *d = dst + (size_t)row * stride;
  for (int k = threadIdx.x % 32; k < A; k += 32) d[pos_of[k]] = s[k];
}
template <typename R>
__global__ void permute_out_host_kernel(const R *__restrict__ src, R *__restrict__ dst,
                                        const int64_t *__restrict__ cell_of,
                                        const int32_t *__restrict__ pos_of, int64_t n, int A,
                                        int stride) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (row >= n) return;
  const R *s = src + (size_t)row * stride;
  R *d = dst + (size_t)cell_of[row] * A;
  for (int k = threadIdx.x % 32; k < A; k += 32) d[k] = s[pos_of[k]];
}

__device__ __forceinline__ double slot_u(const SlotF &s, const double *, int64_t, double x,
                                         double y, double z) {
  return x * (double)s.sx + y * (double)s.sy + z * (double)s.sz - (double)s.w;
}
__device__ __forceinline__ double slot_u(const SlotD &s, const double *wf, int64_t k, double x,
                                         double y, double z) {
  return s.ca * ((x * s.nx + y * s.ny) + z * s.nz) - (wf ? wf[k] : 0.0);
}

// The upwind positivity bound: K = max over cells c and angles a of
// (1/V_c) sum_f max(u_fa, 0); kmax holds it as the bit pattern of a
// non-negative double, which orders like the value.
// The same u in float from float slots (a screening value, error ~1e-7 of
// |cbar A| + |A w|).
__device__ __forceinline__ float slot_u_f(const SlotF &s, const double *, int64_t, float x, float y,
                                          float z) {
  return fmaf(x, s.sx, fmaf(y, s.sy, z * s.sz)) - s.w;
}

// The positivity bound in two passes.  mode 0: the float value of
// K_c = max_a (1/V_c) sum_f max(u_fa, 0) for every cell, max over cells into
// *kf (bits of a non-negative float).  mode 1: every (cell, angle) whose
// float value is within 1e-4 of that maximum is evaluated exactly in double
// and max-ed into *kmax; the float error (~1e-6 of K)
// is far inside the margin, so the maximum found is the exact one (the
// double sum below is the bound's definition, in face order).
template <typename R>
__global__ void positivity_screen_kernel(const int64_t *__restrict__ ptr,
                                         const SlotF *__restrict__ fslot,
                                         const typename SlotOf<R>::type *__restrict__ slot,
                                         const double *__restrict__ wface,
                                         const double *__restrict__ vol,
                                         const double *__restrict__ dir, int64_t n, int A, int mode,
                                         double inv_scale, unsigned *kf,
                                         unsigned long long *kmax, float *kcell) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  float best = 0.0f, braw = 0.0f;  // max over angles of sum / V and of sum
  const float cut = mode == 1 ? __uint_as_float(*kf) * (1.0f - 1e-4f) : 0.0f;
  if (row < n) {
    // fslot holds u scaled by a power of two; 1/V is scaled back by it
    const float iv = (float)(inv_scale / vol[row]);
    for (int a = threadIdx.x % 32; a < A; a += 32) {
      const float x = (float)dir[3 * a], y = (float)dir[3 * a + 1], z = (float)dir[3 * a + 2];
      float sum = 0.0f;
      for (int64_t k = ptr[row]; k < ptr[row + 1]; ++k)
        sum += fmaxf(slot_u_f(fslot[k], nullptr, k, x, y, z), 0.0f);
      const float kc = sum * iv;
      if (mode == 0) {
        best = fmaxf(best, kc);
        braw = fmaxf(braw, sum);
      } else if (kc >= cut) {
        double exact = 0.0;
        for (int64_t k = ptr[row]; k < ptr[row + 1]; ++k) {
          const double u = slot_u(slot[k], wface, k, dir[3 * a], dir[3 * a + 1], dir[3 * a + 2]);
          if (u > 0.0) exact += u;
        }
        atomicMax(kmax, (unsigned long long)__double_as_longlong(exact / vol[row]));
      }
    }
  }
  if (mode == 0) {
    for (int o = 16; o > 0; o >>= 1) {
      best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
      braw = fmaxf(braw, __shfl_xor_sync(0xffffffffu, braw, o));
    }
    if (threadIdx.x % 32 == 0 && row < n) {
      atomicMax(kf, __float_as_uint(best));
      if (kcell) kcell[row] = braw;
    }
  }
}

// Per-cell moments E, F[3], P[6] in double, written in caller order.
template <typename R>
__global__ void moments_kernel(const R *__restrict__ I, const double *__restrict__ dir,
                               const double *__restrict__ wt, const int64_t *__restrict__ cell_of,
                               int64_t n, int A, int stride, double c, double *E, double *F,
                               double *P) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (row >= n) return;
  const R *Ir = I + (size_t)row * stride;
  double s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int a = threadIdx.x % 32; a < A; a += 32) {
    const double wi = wt[a] * (double)Ir[a];
    const double x = dir[3 * a], y = dir[3 * a + 1], z = dir[3 * a + 2];
    s[0] += wi;
    s[1] += wi * x;
    s[2] += wi * y;
    s[3] += wi * z;
    s[4] += wi * x * x;
    s[5] += wi * y * y;
    s[6] += wi * z * z;
    s[7] += wi * x * y;
    s[8] += wi * x * z;
    s[9] += wi * y * z;
  }
#pragma unroll
  for (int k = 0; k < 10; ++k)
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
  if (threadIdx.x % 32) return;
  const int64_t oc = cell_of[row];
  const double fp = 4.0 * kPi;
  if (E) E[oc] = fp * s[0];
  if (F) {
    F[3 * oc] = fp * c * s[1];
    F[3 * oc + 1] = fp * c * s[2];
    F[3 * oc + 2] = fp * c * s[3];
  }
  if (P)
    for (int k = 0; k < 6; ++k) P[6 * oc + k] = fp * s[4 + k];
}

// Totals, pass 1: every block sums a fixed contiguous range of cells in a
// fixed order into partial[block][16].
constexpr int64_t kTotCells = totals_block_cells;  // cells per block of rt_totals
template <typename R>
__global__ void totals_partial_kernel(const R *__restrict__ I, const double *__restrict__ dir,
                                      const double *__restrict__ wt,
                                      const double *__restrict__ vol, const GasDyn *__restrict__ gd,
                                      const double *__restrict__ ext, int64_t n, int A,
                                      int stride, int64_t cpb, double c_over_cbar,
                                      double inv_cbar, double *partial) {
  __shared__ double acc[kThreads / 32][12];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  double t[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  for (int64_t k = warp; k < cpb; k += kThreads / 32) {
    const int64_t row = c0 + k;
    if (row >= n) break;
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
      const GasDyn g = gd[row];
      const double fp = 4.0 * kPi;
      t[0] += V * g.e;
      t[1] += V * c_over_cbar * fp * e;
      t[2] += V * ext[4 * row];
      t[3] += V * g.mx;
      t[4] += V * g.my;
      t[5] += V * g.mz;
      t[6] += V * fp * inv_cbar * fx;  // F / (c cbar) with F = 4 pi c sum w n I
      t[7] += V * fp * inv_cbar * fy;
      t[8] += V * fp * inv_cbar * fz;
      t[9] += V * ext[4 * row + 1];
      t[10] += V * ext[4 * row + 2];
      t[11] += V * ext[4 * row + 3];
    }
  }
  if (lane == 0)
    for (int k = 0; k < 12; ++k) acc[warp][k] = t[k];
  __syncthreads();
  if (threadIdx.x < 12) {
    double s = 0;
    for (int w = 0; w < kThreads / 32; ++w) s += acc[w][threadIdx.x];
    partial[(size_t)blockIdx.x * 12 + threadIdx.x] = s;
  }
}

// Totals, pass 2: component k summed over blocks in block order.
__global__ void totals_final_kernel(const double *__restrict__ partial, int64_t nblocks,
                                    double *out16) {
  const int k = threadIdx.x;
  if (k >= 12) return;
  double s = 0;
  for (int64_t b = 0; b < nblocks; ++b) s += partial[(size_t)b * 12 + k];
  // layout of the public result: 0..2 energy, 3..5 gas m, 6..8 rad, 9..11 ext
  out16[k] = s;
  __syncwarp(0xfffu);
  if (k == 0) out16[12] = out16[0] + out16[1] + out16[2];
  if (k < 3) out16[13 + k] = out16[3 + k] + out16[6 + k] + out16[9 + k];
}

// the inverse of gas_out_kernel for (e, m): caller-order device arrays into
// the internal gas records
__global__ void gas_in_kernel(const double *__restrict__ e, const double *__restrict__ m,
                              const int64_t *__restrict__ cell_of, int64_t n, GasDyn *gd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t oc = cell_of[i];
  gd[i] = GasDyn{e[oc], m[3 * oc], m[3 * oc + 1], m[3 * oc + 2]};
}

__global__ void gas_out_kernel(const GasDyn *__restrict__ gd, const double *__restrict__ ext,
                               const int64_t *__restrict__ cell_of, int64_t n, double *e,
                               double *m, double *x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t oc = cell_of[i];
  const GasDyn g = gd[i];
  if (e) e[oc] = g.e;
  if (m) {
    m[3 * oc] = g.mx;
    m[3 * oc + 1] = g.my;
    m[3 * oc + 2] = g.mz;
  }
  if (x)
    for (int k = 0; k < 4; ++k) x[4 * oc + k] = ext[4 * i + k];
}

// cellv = (m / rho, e - |m|^2 / (2 rho)) in the state precision, as the step
// kernel's gas update writes it
template <typename R>
__global__ void cellv_kernel(const GasStatic *__restrict__ gs, const GasDyn *__restrict__ gd,
                             int64_t n, R *cellv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const GasStatic g = gs[i];
  const GasDyn d = gd[i];
  const double ir = g.inv_rho;
  cellv[4 * i] = R(d.mx * ir);
  cellv[4 * i + 1] = R(d.my * ir);
  cellv[4 * i + 2] = R(d.mz * ir);
  cellv[4 * i + 3] = R(d.e - 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * ir);
}

unsigned rows_grid(int64_t n) { return (unsigned)((n + kThreads / 32 - 1) / (kThreads / 32)); }
// the device permutes: two rows per warp iteration, at most 16 blocks per SM
// worth of warps (the loop strides over the rest)
unsigned permute_grid(int64_t n) {
  const int64_t blocks = (n + 2 * (kThreads / 32) - 1) / (2 * (kThreads / 32));
  return (unsigned)(blocks < 152 * 16 ? (blocks > 0 ? blocks : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_permute_in(rt_state *s, const void *src, void *dst, int stride) {
  if (s->precision == RT_FP32)
    permute_in_kernel<float><<<permute_grid(s->n_cells), kThreads, 0, s->stream>>>(
        (const float *)src, (float *)dst, s->d_cell_of, s->d_angle_of, s->n_cells, s->n_angles,
        stride);
  else
    permute_in_kernel<double><<<permute_grid(s->n_cells), kThreads, 0, s->stream>>>(
        (const double *)src, (double *)dst, s->d_cell_of, s->d_angle_of, s->n_cells,
        s->n_angles, stride);
  s->launches++;
  return cudaGetLastError();
}

cudaError_t launch_permute_out(rt_state *s, const void *src, void *dst, int stride) {
  if (s->precision == RT_FP32)
    permute_out_kernel<float><<<permute_grid(s->n_cells), kThreads, 0, s->stream>>>(
        (const float *)src, (float *)dst, s->d_cell_of, s->d_angle_of, s->n_cells, s->n_angles,
        stride);
  else
    permute_out_kernel<double><<<permute_grid(s->n_cells), kThreads, 0, s->stream>>>(
        (const double *)src, (double *)dst, s->d_cell_of, s->d_angle_of, s->n_cells,
        s->n_angles, stride);
  s->launches++;
  return cudaGetLastError();
}

cudaError_t launch_permute_in_host(rt_state *s, const void *src, void *dst, int stride) {
  if (s->precision == RT_FP32)
    permute_in_host_kernel<float><<<rows_grid(s->n_cells), kThreads, 0, s->stream>>>(
        (const float *)src, (float *)dst, s->d_cell_of, s->d_pos_of, s->n_cells, s->n_angles,
        stride);
  else
    permute_in_host_kernel<double><<<rows_grid(s->n_cells), kThreads, 0, s->stream>>>(
        (const double *)src, (double *)dst, s->d_cell_of, s->d_pos_of, s->n_cells, s->n_angles,
        stride);
  s->launches++;
  return cudaGetLastError();
}

cudaError_t launch_permute_out_host(rt_state *s, const void *src, void *dst, int stride) {
  if (s->precision == RT_FP32)
    permute_out_host_kernel<float><<<rows_grid(s->n_cells), kThreads, 0, s->stream>>>(
        (const float *)src, (float *)dst, s->d_cell_of, s->d_pos_of, s->n_cells, s->n_angles,
        stride);
  else
    permute_out_host_kernel<double><<<rows_grid(s->n_cells), kThreads, 0, s->stream>>>(
        (const double *)src, (double *)dst, s->d_cell_of, s->d_pos_of, s->n_cells, s->n_angles,
        stride);
  s->launches++;
  return cudaGetLastError();
}

// d_kmax[0] receives the bound (as a double), d_kmax[1] is scratch.
// fslot: the face slots in float (the state's own for float states).
cudaError_t launch_positivity(rt_state *s, const SlotF *fslot, double *d_kmax, float *kcell) {
  cudaError_t e = cudaMemsetAsync(d_kmax, 0, 2 * sizeof(double), s->stream);
  if (e != cudaSuccess) return e;
  unsigned *kf = reinterpret_cast<unsigned *>(d_kmax + 1);
  unsigned long long *km = reinterpret_cast<unsigned long long *>(d_kmax);
  for (int mode = 0; mode < 2; ++mode) {
    if (s->precision == RT_FP32)
      positivity_screen_kernel<float><<<rows_grid(s->n_cells), kThreads, 0, s->stream>>>(
          s->d_ptr, fslot, (const SlotF *)s->d_slot, s->d_wface, s->d_volume, s->d_dir64,
          s->n_cells, s->n_angles, mode, 1.0 / s->screen_scale, kf, km, kcell);
    else
      positivity_screen_kernel<double><<<rows_grid(s->n_cells), kThreads, 0, s->stream>>>(
          s->d_ptr, fslot, (const SlotD *)s->d_slot, s->d_wface, s->d_volume, s->d_dir64,
          s->n_cells, s->n_angles, mode, 1.0 / s->screen_scale, kf, km, kcell);
    s->launches++;
  }
  return cudaGetLastError();
}

cudaError_t launch_moments(rt_state *s, double *E, double *F, double *P) {
  const void *I = s->d_I[s->cur];
  if (s->precision == RT_FP32)
    moments_kernel<float><<<rows_grid(s->n_cells), kThreads, 0, s->stream>>>(
        (const float *)I, s->d_dir64, s->d_wt64, s->d_cell_of, s->n_cells, s->n_angles,
        s->row_stride, s->params.c, E, F, P);
  else
    moments_kernel<double><<<rows_grid(s->n_cells), kThreads, 0, s->stream>>>(
        (const double *)I, s->d_dir64, s->d_wt64, s->d_cell_of, s->n_cells, s->n_angles,
        s->row_stride, s->params.c, E, F, P);
  s->launches++;
  return cudaGetLastError();
}

cudaError_t launch_totals_with(rt_state *s, double *partial, int64_t cpb, double *d_out16) {
  const int64_t nb = (s->n_cells + cpb - 1) / cpb;
  const void *I = s->d_I[s->cur];
  const double coc = s->params.c / s->params.cbar, icb = 1.0 / s->params.cbar;
  if (s->precision == RT_FP32)
    totals_partial_kernel<float><<<(unsigned)nb, kThreads, 0, s->stream>>>(
        (const float *)I, s->d_dir64, s->d_wt64, s->d_volume, s->d_gd, s->d_ext, s->n_cells,
        s->n_angles, s->row_stride, cpb, coc, icb, partial);
  else
    totals_partial_kernel<double><<<(unsigned)nb, kThreads, 0, s->stream>>>(
        (const double *)I, s->d_dir64, s->d_wt64, s->d_volume, s->d_gd, s->d_ext, s->n_cells,
        s->n_angles, s->row_stride, cpb, coc, icb, partial);
  totals_final_kernel<<<1, 32, 0, s->stream>>>(partial, nb, d_out16);
  s->launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_totals(rt_state *s, double *d_out16) {
  const int64_t nb = (s->n_cells + kTotCells - 1) / kTotCells;
  if ((size_t)nb * 12 > s->scratch_len) return cudaErrorInvalidValue;
  return launch_totals_with(s, s->d_scratch, kTotCells, d_out16);
}

int64_t totals_scratch_len(int64_t n_cells) { return ((n_cells + kTotCells - 1) / kTotCells) * 12; }

cudaError_t launch_gas_in(rt_state *s, const double *e, const double *m) {
  const unsigned g = (unsigned)((s->n_cells + kThreads - 1) / kThreads);
  gas_in_kernel<<<g, kThreads, 0, s->stream>>>(e, m, s->d_cell_of, s->n_cells, s->d_gd);
  s->launches++;
  return cudaGetLastError();
}

cudaError_t launch_gas_out(rt_state *s, double *e, double *m, double *ext) {
  gas_out_kernel<<<(unsigned)((s->n_cells + kThreads - 1) / kThreads), kThreads, 0, s->stream>>>(
      s->d_gd, s->d_ext, s->d_cell_of, s->n_cells, e, m, ext);
  s->launches++;
  return cudaGetLastError();
}

template <typename R>
__global__ void inv_vol_kernel(const double *__restrict__ vol, R *__restrict__ inv, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) inv[i] = (R)(1.0 / vol[i]);
}

cudaError_t launch_inv_vol(rt_state *s) {
  const unsigned g = (unsigned)((s->n_cells + kThreads - 1) / kThreads);
  if (s->precision == RT_FP32)
    inv_vol_kernel<float><<<g, kThreads, 0, s->stream>>>(s->d_volume, (float *)s->d_inv_vol,
                                                         s->n_cells);
  else
    inv_vol_kernel<double><<<g, kThreads, 0, s->stream>>>(s->d_volume, (double *)s->d_inv_vol,
                                                          s->n_cells);
  s->launches++;
  return cudaGetLastError();
}

// rho kappa_J(T) = rkJ0 (T / T_ref)^beta_J at each cell's gas temperature
// (the same expression the step's gas phase evaluates for the next step).
__global__ void opacity_refresh_kernel(GasStatic *__restrict__ gs, const GasDyn *__restrict__ gd,
                                       const double *__restrict__ rkJ0, int64_t n, double beta_J,
                                       double T_ref) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const GasDyn d = gd[i];
  const double kin = 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * gs[i].inv_rho;
  const double rkJ = rkJ0[i] * pow((d.e - kin) / gs[i].rcv / T_ref, beta_J);
  gs[i].rkJ = rkJ;
  gs[i].frkJ = (float)rkJ;
}

cudaError_t launch_opacity_refresh(rt_state *s) {
  if (s->params.beta_J == 0.0 || !s->d_rkJ0) return cudaSuccess;
  const unsigned g = (unsigned)((s->n_cells + kThreads - 1) / kThreads);
  opacity_refresh_kernel<<<g, kThreads, 0, s->stream>>>(s->d_gs, s->d_gd, s->d_rkJ0, s->n_cells,
                                                        s->params.beta_J, s->params.T_ref);
  s->launches++;
  return cudaGetLastError();
}

cudaError_t launch_cellv(rt_state *s) {
  const unsigned g = (unsigned)((s->n_cells + kThreads - 1) / kThreads);
  if (s->precision == RT_FP32)
    cellv_kernel<float><<<g, kThreads, 0, s->stream>>>(s->d_gs, s->d_gd, s->n_cells,
                                                       (float *)s->d_cellv);
  else
    cellv_kernel<double><<<g, kThreads, 0, s->stream>>>(s->d_gs, s->d_gd, s->n_cells,
                                                        (double *)s->d_cellv);
  s->launches++;
  return cudaGetLastError();
}

}  // namespace rt
