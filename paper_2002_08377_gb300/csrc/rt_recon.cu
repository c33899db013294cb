// Limited linear reconstruction and the van Leer step (Sec. 2, integration
// steps with the van Leer half step; Sec. 2.2, transport step 2: the face
// state by linear reconstruction with a limiter).
//
// One step of the van Leer integrator is four launches:
//   1. the fused step kernel over dt/2 from I^n into I^{n+1/2} (first-order
//      upwinding), its gas update discarded;
//   2. gradient_kernel: least-squares gradients of I^{n+1/2} over each cell's
//      face neighbours, weights A_f / |r_f|^2, limited (Barth-Jespersen) so
//      that the reconstructed face values stay within the range of the cell
//      and its neighbours;
//   3. recon_transport_kernel: I* = I^n - dt/V sum_f u I_up with the upwind
//      value reconstructed at the face centre from I^{n+1/2} and its gradient
//      (the same value on both sides of a face, so the update conserves);
//   4. the fused step kernel in source-only mode over dt from the gas at n.
// The paper defers the gradient estimate and the limiter to its hydro code;
// these are the readings the oracle uses too.
#include <cuda_runtime.h>

#include "rt_internal.cuh"
#include "rt_step_common.cuh"

namespace rt {
namespace {
using namespace step;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ float rmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double rmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float rmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double rmax(double a, double b) { return fmax(a, b); }

// grad[(c * 3 + d) * RS + q]: limited gradient of the intensity at row
// position q of cell c.  recon[8 k] = (x_f - x_c, w_f, x_f - x_nbr', 0) of
// slot k; lsq[8 c] = the inverse of sum_f w_f r_f r_f^T (xx, xy, xz, yy, yz,
// zz).  One warp per cell, lanes over row positions.
template <typename R>
__global__ void __launch_bounds__(kThreads) gradient_kernel(
    const int64_t *__restrict__ ptr, const int32_t *__restrict__ nbr, const R *__restrict__ recon,
    const R *__restrict__ lsq, const R *__restrict__ Ih, R *__restrict__ grad, int64_t n, int A,
    int RS) {
  const int64_t c = (int64_t)blockIdx.x * kWarps + threadIdx.x / 32;
  if (c >= n) return;
  const int lane = threadIdx.x % 32;
  const R *L = lsq + 8 * c;
  const R m00 = L[0], m01 = L[1], m02 = L[2], m11 = L[3], m12 = L[4], m22 = L[5];
  const int64_t k0 = ptr[c], k1 = ptr[c + 1];
  for (int q = lane; q < A; q += 32) {
    const R Ic = Ih[(size_t)c * RS + q];
    R bx = 0, by = 0, bz = 0, lo = Ic, hi = Ic;
    for (int64_t k = k0; k < k1; ++k) {
      const R *g = recon + 8 * k;
      const R w = g[3];
      const R Ij = Ih[(size_t)nbr[k] * RS + q];
      const R d = Ij - Ic;
      bx += w * (g[0] - g[4]) * d;
      by += w * (g[1] - g[5]) * d;
      bz += w * (g[2] - g[6]) * d;
      lo = rmin(lo, Ij);
      hi = rmax(hi, Ij);
    }
    const R gx = m00 * bx + m01 * by + m02 * bz;
    const R gy = m01 * bx + m11 * by + m12 * bz;
    const R gz = m02 * bx + m12 * by + m22 * bz;
    R alpha = 1;
    for (int64_t k = k0; k < k1; ++k) {
      const R *g = recon + 8 * k;
      const R dI = gx * g[0] + gy * g[1] + gz * g[2];
      R al = 1;
      if (dI > R(0))
        al = (hi - Ic) / dI;
      else if (dI < R(0))
        al = (lo - Ic) / dI;
      alpha = rmin(alpha, al);
    }
    R *o = grad + (size_t)c * 3 * RS + q;
    o[0] = alpha * gx;
    o[RS] = alpha * gy;
    o[2 * (size_t)RS] = alpha * gz;
  }
}

// Flux coefficient u of row position q (angle a = angle_of[q]) through slot
// k, exactly as the fused step kernel forms it: float from the slot and the
// direction, double from the tabulated n_p . s (the antipode's is its
// negative); minus A w . n on a moving mesh.
template <bool MOVING>
__device__ __forceinline__ float flux_coef(const SlotF *slot, const double *, const double *,
                                           int64_t k, int, float nx, float ny, float nz, int, bool) {
  const SlotF s = slot[k];
  const float d = fmaf(nx, s.sx, fmaf(ny, s.sy, nz * s.sz));
  return MOVING ? d - s.w : d;
}
template <bool MOVING>
__device__ __forceinline__ double flux_coef(const SlotD *, const double *wface, const double *uface,
                                            int64_t k, int H, double, double, double, int p,
                                            bool anti) {
  const double d = uface[(size_t)k * H + p];
  const double u = anti ? -d : d;
  return MOVING ? u - wface[k] : u;
}

// I*[c][q] = I[c][q] - dt / V_c sum_f u I_up, I_up reconstructed at the face
// centre from (Ih, grad) of the upwind cell.  One warp per cell.
template <typename R, bool MOVING>
__global__ void __launch_bounds__(kThreads) recon_transport_kernel(
    const int64_t *__restrict__ ptr, const int32_t *__restrict__ nbr,
    const typename SlotOf<R>::type *__restrict__ slot, const double *__restrict__ wface,
    const double *__restrict__ uface, const R *__restrict__ recon, const R *__restrict__ dir,
    const int32_t *__restrict__ angle_of, const R *__restrict__ inv_vol, const R *__restrict__ I,
    const R *__restrict__ Ih, const R *__restrict__ grad, R *__restrict__ Istar, int64_t n, int A,
    int RS, R dt) {
  const int64_t c = (int64_t)blockIdx.x * kWarps + threadIdx.x / 32;
  if (c >= n) return;
  const int lane = threadIdx.x % 32, H = A / 2;
  const int64_t k0 = ptr[c], k1 = ptr[c + 1];
  const size_t gs = (size_t)RS;
  for (int q = lane; q < A; q += 32) {
    const int a = angle_of[q];
    const bool anti = a >= H;
    const int p = anti ? a - H : a;
    const R nx = dir[4 * a], ny = dir[4 * a + 1], nz = dir[4 * a + 2];
    const R Ihc = Ih[(size_t)c * RS + q];
    const R *gc = grad + (size_t)c * 3 * gs + q;
    const R gcx = gc[0], gcy = gc[gs], gcz = gc[2 * gs];
    R acc = 0;
    for (int64_t k = k0; k < k1; ++k) {
      const R u = flux_coef<MOVING>(slot, wface, uface, k, H, nx, ny, nz, p, anti);
      const R *g = recon + 8 * k;
      if (positive(u)) {
        acc += u * (Ihc + (gcx * g[0] + gcy * g[1] + gcz * g[2]));
      } else if (u < R(0)) {
        const int64_t j = nbr[k];
        const R *gj = grad + (size_t)j * 3 * gs + q;
        acc += u * (Ih[(size_t)j * RS + q] + (gj[0] * g[4] + gj[gs] * g[5] + gj[2 * gs] * g[6]));
      }
    }
    Istar[(size_t)c * RS + q] = I[(size_t)c * RS + q] - dt * inv_vol[c] * acc;
  }
}

unsigned warp_grid(int64_t n) { return (unsigned)((n + kWarps - 1) / kWarps); }

template <typename R> cudaError_t vl_middle(rt_state *s, double dt) {
  const int64_t N = s->n_cells;
  const int A = s->n_angles, RS = s->row_stride;
  const R *recon = reinterpret_cast<const R *>(s->d_recon);
  const R *Ih = reinterpret_cast<const R *>(s->d_Ihalf);
  R *grad = reinterpret_cast<R *>(s->d_grad);
  gradient_kernel<R><<<warp_grid(N), kThreads, 0, s->stream>>>(
      s->d_ptr, s->d_nbr, recon, reinterpret_cast<const R *>(s->d_lsq), Ih, grad, N, A, RS);
  const auto *slot = reinterpret_cast<const typename SlotOf<R>::type *>(s->d_slot);
  const R *dir = reinterpret_cast<const R *>(s->d_dir);
  const R *iv = reinterpret_cast<const R *>(s->d_inv_vol);
  const R *I = reinterpret_cast<const R *>(s->d_I[s->cur]);
  R *Is = reinterpret_cast<R *>(s->d_I[s->cur ^ 1]);
  if (s->moving)
    recon_transport_kernel<R, true><<<warp_grid(N), kThreads, 0, s->stream>>>(
        s->d_ptr, s->d_nbr, slot, s->d_wface, s->d_uface, recon, dir, s->d_angle_of, iv, I, Ih,
        grad, Is, N, A, RS, R(dt));
  else
    recon_transport_kernel<R, false><<<warp_grid(N), kThreads, 0, s->stream>>>(
        s->d_ptr, s->d_nbr, slot, s->d_wface, s->d_uface, recon, dir, s->d_angle_of, iv, I, Ih,
        grad, Is, N, A, RS, R(dt));
  s->launches += 2;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_vl(rt_state *s, double dt) {
  // stage 1: first-order step over dt/2 into the half buffer, gas discarded
  const StepIO half{s->d_I[s->cur], s->d_Ihalf, false, false};
  cudaError_t e = launch_step_io(s, 0.5 * dt, half);
  if (e != cudaSuccess) return e;
  // stage 2: reconstructed fluxes of I^{n+1/2} applied to I^n (into the
  // output buffer), then the source over dt in place
  e = (s->precision == RT_FP32) ? vl_middle<float>(s, dt) : vl_middle<double>(s, dt);
  if (e != cudaSuccess) return e;
  const StepIO src{s->d_I[s->cur ^ 1], s->d_I[s->cur ^ 1], true, true};
  return launch_step_io(s, dt, src);
}

}  // namespace rt
