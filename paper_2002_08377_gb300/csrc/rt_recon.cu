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

// The stage-1 intensity and its limited gradient of one row position,
// stored together so that the transport fetches them with one access:
// IG[(c * RS + q)] = (I, g_x, g_y, g_z).
template <typename R> struct QV;
template <> struct QV<float> {
  float i, x, y, z;
  __device__ static QV load(const float *p) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return {v.x, v.y, v.z, v.w};
  }
  __device__ void store(float *p) const {
    *reinterpret_cast<float4 *>(p) = make_float4(i, x, y, z);
  }
};
template <> struct QV<double> {
  double i, x, y, z;
  __device__ static QV load(const double *p) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return {a.x, a.y, b.x, b.y};
  }
  __device__ void store(double *p) const {
    reinterpret_cast<double2 *>(p)[0] = make_double2(i, x);
    reinterpret_cast<double2 *>(p)[1] = make_double2(y, z);
  }
};

// Per warp, a cell's face geometry is staged in shared memory CH slots at a
// time: recon (x_f - x_c, w_f, x_f - x_nbr', 0), the neighbour index and,
// for the float transport, the face slot (c A n, A w.n).
constexpr int CH = 32;
template <typename R> struct WarpStage {
  R geo[CH][8];
  SlotF slot[CH];
  int32_t nb[CH];
};

// Copies slots [k, k + cnt) of the cell into the warp's stage (cnt <= CH).
template <typename R>
__device__ __forceinline__ void stage_faces(WarpStage<R> &st, const R *__restrict__ recon,
                                            const int32_t *__restrict__ nbr, const SlotF *slotf,
                                            int64_t k, int cnt, int lane) {
  for (int l = lane; l < cnt; l += 32) {
    const R *g = recon + 8 * (k + l);
#pragma unroll
    for (int x = 0; x < 8; ++x) st.geo[l][x] = g[x];
    st.nb[l] = nbr[k + l];
    if (slotf) st.slot[l] = slotf[k + l];
  }
  __syncwarp();
}

// IG[c * RS + q] = (I, limited gradient) of the stage-1 intensity at row
// position q of cell c (lsq[8 c] = the inverse of sum_f w_f r_f r_f^T as
// xx, xy, xz, yy, yz, zz).  One warp per cell; lane l takes the positions
// l + 32 i (i < QN).  The limiter factor is the oracle's min over faces
// of (max - I_c) / d_f (d_f > 0) and (min - I_c) / d_f (d_f < 0), taken as one
// division by the largest and one by the smallest d_f: correctly rounded
// division is monotone in d_f, so the result is the same number.
template <typename R, int QN>
__global__ void __launch_bounds__(kThreads) gradient_kernel(
    const int64_t *__restrict__ ptr, const int32_t *__restrict__ nbr, const R *__restrict__ recon,
    const R *__restrict__ lsq, const R *__restrict__ Ih, R *__restrict__ IG, int64_t n, int A,
    int RS) {
  __shared__ WarpStage<R> stage[kWarps];
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t c = (int64_t)blockIdx.x * kWarps + w;
  if (c >= n) return;
  WarpStage<R> &st = stage[w];
  const int64_t k0 = ptr[c], k1 = ptr[c + 1];
  R Ic[QN], bx[QN], by[QN], bz[QN], lo[QN], hi[QN];
#pragma unroll
  for (int i = 0; i < QN; ++i) {
    const int q = lane + 32 * i;
    Ic[i] = q < A ? Ih[(size_t)c * RS + q] : R(0);
    lo[i] = hi[i] = Ic[i];
    bx[i] = by[i] = bz[i] = R(0);
  }
  for (int64_t kc = k0; kc < k1; kc += CH) {
    const int cnt = (int)(k1 - kc < CH ? k1 - kc : CH);
    stage_faces<R>(st, recon, nbr, nullptr, kc, cnt, lane);
    for (int t = 0; t < cnt; ++t) {
      const R *g = st.geo[t];
      const R rx = g[0] - g[4], ry = g[1] - g[5], rz = g[2] - g[6], wt = g[3];
      const R *row = Ih + (size_t)st.nb[t] * RS;
#pragma unroll
      for (int i = 0; i < QN; ++i) {
        const int q = lane + 32 * i;
        if (q < A) {
          const R Ij = row[q];
          const R d = Ij - Ic[i];
          bx[i] += wt * rx * d;
          by[i] += wt * ry * d;
          bz[i] += wt * rz * d;
          lo[i] = rmin(lo[i], Ij);
          hi[i] = rmax(hi[i], Ij);
        }
      }
    }
    __syncwarp();
  }
  const R *L = lsq + 8 * c;
  const R m00 = L[0], m01 = L[1], m02 = L[2], m11 = L[3], m12 = L[4], m22 = L[5];
  R gx[QN], gy[QN], gz[QN], dmax[QN], dmin[QN];
#pragma unroll
  for (int i = 0; i < QN; ++i) {
    gx[i] = m00 * bx[i] + m01 * by[i] + m02 * bz[i];
    gy[i] = m01 * bx[i] + m11 * by[i] + m12 * bz[i];
    gz[i] = m02 * bx[i] + m12 * by[i] + m22 * bz[i];
    dmax[i] = dmin[i] = R(0);
  }
  for (int64_t kc = k0; kc < k1; kc += CH) {
    const int cnt = (int)(k1 - kc < CH ? k1 - kc : CH);
    if (k1 - k0 > CH) stage_faces<R>(st, recon, nbr, nullptr, kc, cnt, lane);
    for (int t = 0; t < cnt; ++t) {
      const R *g = st.geo[t];
#pragma unroll
      for (int i = 0; i < QN; ++i) {
        const R dI = gx[i] * g[0] + gy[i] * g[1] + gz[i] * g[2];
        dmax[i] = rmax(dmax[i], dI);
        dmin[i] = rmin(dmin[i], dI);
      }
    }
    if (k1 - k0 > CH) __syncwarp();
  }
#pragma unroll
  for (int i = 0; i < QN; ++i) {
    const int q = lane + 32 * i;
    if (q < A) {
      R alpha = 1;
      if (dmax[i] > R(0)) alpha = rmin(alpha, (hi[i] - Ic[i]) / dmax[i]);
      if (dmin[i] < R(0)) alpha = rmin(alpha, (lo[i] - Ic[i]) / dmin[i]);
      const QV<R> v{Ic[i], alpha * gx[i], alpha * gy[i], alpha * gz[i]};
      v.store(IG + 4 * ((size_t)c * RS + q));
    }
  }
}

// I*[c][q] = I[c][q] - dt / V_c sum_f u I_up, I_up reconstructed at the face
// centre from IG of the upwind cell.  u as the fused step kernel forms it:
// float from the face slot and the angle's direction, double from the
// tabulated n_p . s (negated for the antipode); minus A w . n on a moving
// mesh.  One warp per cell, lane l takes positions l + 32 i (i < QN); every
// lane fetches the neighbour's record and selects the upwind value, so the
// warp does not diverge per face.
template <typename R, bool MOVING, int QN>
__global__ void __launch_bounds__(kThreads) recon_transport_kernel(
    const int64_t *__restrict__ ptr, const int32_t *__restrict__ nbr, const SlotF *__restrict__ slotf,
    const double *__restrict__ wface, const double *__restrict__ uface, const R *__restrict__ recon,
    const R *__restrict__ dir, const int32_t *__restrict__ angle_of, const R *__restrict__ inv_vol,
    const R *__restrict__ I, const R *__restrict__ IG, R *__restrict__ Istar, int64_t n, int A,
    int RS, R dt) {
  __shared__ WarpStage<R> stage[kWarps];
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t c = (int64_t)blockIdx.x * kWarps + w;
  if (c >= n) return;
  WarpStage<R> &st = stage[w];
  const int H = A / 2;
  const int64_t k0 = ptr[c], k1 = ptr[c + 1];
  R nx[QN], ny[QN], nz[QN], acc[QN];
  QV<R> own[QN];
  int pp[QN], qq[QN];
  bool anti[QN];
#pragma unroll
  for (int i = 0; i < QN; ++i) {
    const int q = lane + 32 * i;
    qq[i] = q < A ? q : A - 1;  // idle lanes shadow the last position
    const int a = angle_of[qq[i]];
    anti[i] = a >= H;
    pp[i] = anti[i] ? a - H : a;
    nx[i] = dir[4 * a];
    ny[i] = dir[4 * a + 1];
    nz[i] = dir[4 * a + 2];
    own[i] = QV<R>::load(IG + 4 * ((size_t)c * RS + qq[i]));
    acc[i] = R(0);
  }
  for (int64_t kc = k0; kc < k1; kc += CH) {
    const int cnt = (int)(k1 - kc < CH ? k1 - kc : CH);
    stage_faces<R>(st, recon, nbr, sizeof(R) == 4 ? slotf : nullptr, kc, cnt, lane);
    for (int t = 0; t < cnt; ++t) {
      const R *g = st.geo[t];
      const R *IGj = IG + 4 * (size_t)st.nb[t] * RS;
      R wk = R(0);
      if (MOVING) wk = sizeof(R) == 4 ? R(st.slot[t].w) : R(wface[kc + t]);
      SlotF sl{0, 0, 0, 0};
      if constexpr (sizeof(R) == 4) sl = st.slot[t];
#pragma unroll
      for (int i = 0; i < QN; ++i) {
        R d;
        if constexpr (sizeof(R) == 4) {
          d = fmaf(nx[i], sl.sx, fmaf(ny[i], sl.sy, nz[i] * sl.sz));
        } else {
          const R dd = uface[(size_t)(kc + t) * H + pp[i]];
          d = anti[i] ? -dd : dd;
        }
        const R u = MOVING ? d - wk : d;
        const QV<R> nb = QV<R>::load(IGj + 4 * qq[i]);
        const R vo = own[i].i + (own[i].x * g[0] + own[i].y * g[1] + own[i].z * g[2]);
        const R vn = nb.i + (nb.x * g[4] + nb.y * g[5] + nb.z * g[6]);
        // u = 0 carries no flux: either value times zero
        acc[i] += u * (positive(u) ? vo : vn);
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int i = 0; i < QN; ++i) {
    const int q = lane + 32 * i;
    if (q < A) Istar[(size_t)c * RS + q] = I[(size_t)c * RS + q] - dt * inv_vol[c] * acc[i];
  }
}

unsigned warp_grid(int64_t n) { return (unsigned)((n + kWarps - 1) / kWarps); }

template <typename R, int QN> cudaError_t vl_middle_q(rt_state *s, double dt) {
  const int64_t N = s->n_cells;
  const int A = s->n_angles, RS = s->row_stride;
  const R *recon = reinterpret_cast<const R *>(s->d_recon);
  const R *Ih = reinterpret_cast<const R *>(s->d_Ihalf);
  R *IG = reinterpret_cast<R *>(s->d_grad);
  gradient_kernel<R, QN><<<warp_grid(N), kThreads, 0, s->stream>>>(
      s->d_ptr, s->d_nbr, recon, reinterpret_cast<const R *>(s->d_lsq), Ih, IG, N, A, RS);
  const SlotF *slotf = sizeof(R) == 4 ? reinterpret_cast<const SlotF *>(s->d_slot) : nullptr;
  const R *dir = reinterpret_cast<const R *>(s->d_dir);
  const R *iv = reinterpret_cast<const R *>(s->d_inv_vol);
  const R *I = reinterpret_cast<const R *>(s->d_I[s->cur]);
  R *Is = reinterpret_cast<R *>(s->d_I[s->cur ^ 1]);
  if (s->moving)
    recon_transport_kernel<R, true, QN><<<warp_grid(N), kThreads, 0, s->stream>>>(
        s->d_ptr, s->d_nbr, slotf, s->d_wface, s->d_uface, recon, dir, s->d_angle_of, iv, I, IG, Is,
        N, A, RS, R(dt));
  else
    recon_transport_kernel<R, false, QN><<<warp_grid(N), kThreads, 0, s->stream>>>(
        s->d_ptr, s->d_nbr, slotf, s->d_wface, s->d_uface, recon, dir, s->d_angle_of, iv, I, IG, Is,
        N, A, RS, R(dt));
  s->launches += 2;
  return cudaGetLastError();
}

template <typename R> cudaError_t vl_middle(rt_state *s, double dt) {
  switch ((s->n_angles + 31) / 32) {
    case 1: return vl_middle_q<R, 1>(s, dt);
    case 2: return vl_middle_q<R, 2>(s, dt);
    case 3: return vl_middle_q<R, 3>(s, dt);
    case 4: return vl_middle_q<R, 4>(s, dt);
    default: return cudaErrorInvalidValue;
  }
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
