// Discrete adjoint of one radiation step (transport, Sec. 2.2, then the
// implicit comoving source, Sec. 2.3), for gradients of a scalar loss with
// respect to the per-cell absorption opacities and the initial intensities.
//
//   I*  = M I^n                       (linear upwind transport)
//   (I^{n+1}, e^{n+1}, m^{n+1}) = S(I*, e^n, m^n; kappa_P, kappa_J)
//
// Reverse: the source adjoint per cell gives dL/dI*, dL/de^n, dL/dm^n and
// accumulates dL/dkappa; the transport adjoint is M^T applied by a gather
// over the same face lists.  The temperature T^{n+1} is defined implicitly
// by alpha T^4 + rho c_v T - g = 0; its derivatives follow from the
// implicit-function theorem, dT/dalpha = -T^4 / F', dT/dg = 1 / F',
// F' = 4 alpha T^3 + rho c_v.  The source adjoint runs in double for both
// state precisions (one warp per cell, lanes over angles); it is not on the
// forward hot path.
#include <cuda_runtime.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxPerLane = 4;  // angles per lane: A <= 128

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float slot_u(const SlotF &s, const double *, int64_t, float x, float y,
                                        float z) {
  return fmaf(x, s.sx, fmaf(y, s.sy, z * s.sz)) - s.w;
}
__device__ __forceinline__ double slot_u(const SlotD &s, const double *wf, int64_t k, double x,
                                         double y, double z) {
  const double d = __dmul_rn(s.ca, __dadd_rn(__dadd_rn(__dmul_rn(x, s.nx), __dmul_rn(y, s.ny)),
                                            __dmul_rn(z, s.nz)));
  return d - (wf ? wf[k] : 0.0);
}


// I* = I - dt/V sum_f u I_up, one warp per cell, lanes over caller angles
// (the same face order and flux coefficient as the fused step kernel).
template <typename R>
__global__ void transport_kernel(const int64_t *__restrict__ ptr, const int32_t *__restrict__ nbr,
                                 const typename SlotOf<R>::type *__restrict__ slot,
                                 const double *__restrict__ wface, const R *__restrict__ inv_vol,
                                 const R *__restrict__ dir, const R *__restrict__ I, R *__restrict__ Is,
                                 int64_t n, int A, int quad_end, R dt) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (c >= n) return;
  const int lane = threadIdx.x % 32, H = A / 2;
  for (int a = lane; a < A; a += 32) {
    const R x = dir[4 * a], y = dir[4 * a + 1], z = dir[4 * a + 2];
    const int q = position_of_angle(a, H, quad_end);
    const R own = I[(size_t)c * A + q];
    R acc = 0;
    for (int64_t k = ptr[c]; k < ptr[c + 1]; ++k) {
      const R u = slot_u(slot[k], wface, k, x, y, z);
      const R up = u > R(0) ? own : I[(size_t)nbr[k] * A + q];
      acc = fma(u, up, acc);
    }
    Is[(size_t)c * A + q] = fma(-dt * inv_vol[c], acc, own);
  }
}

// (M^T l)_ja = l_ja - sum_{f in j, u_jfa > 0} u_jfa (dt/V_j l_ja - dt/V_nbr l_nbr,a)
template <typename R>
__global__ void transport_adjoint_kernel(const int64_t *__restrict__ ptr,
                                         const int32_t *__restrict__ nbr,
                                         const typename SlotOf<R>::type *__restrict__ slot,
                                         const double *__restrict__ wface,
                                         const R *__restrict__ inv_vol, const R *__restrict__ dir,
                                         const R *__restrict__ l, R *__restrict__ out, int64_t n,
                                         int A, int quad_end, R dt) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (c >= n) return;
  const int lane = threadIdx.x % 32, H = A / 2;
  const R dvc = dt * inv_vol[c];
  for (int a = lane; a < A; a += 32) {
    const R x = dir[4 * a], y = dir[4 * a + 1], z = dir[4 * a + 2];
    const int q = position_of_angle(a, H, quad_end);
    const R own = l[(size_t)c * A + q];
    R acc = 0;
    for (int64_t k = ptr[c]; k < ptr[c + 1]; ++k) {
      const R u = slot_u(slot[k], wface, k, x, y, z);
      if (u > R(0)) {
        const int32_t j = nbr[k];
        acc = fma(u, dvc * own - dt * inv_vol[j] * l[(size_t)j * A + q], acc);
      }
    }
    out[(size_t)c * A + q] = own - acc;
  }
}

struct SrcAdjArgs {
  int64_t n;
  int A;
  const GasStatic *gs;
  const uint8_t *kind;
  const double2 *aux;
  const double *dir;   // [A][3] internal angle order, double
  const double *wt;    // [A] internal angle order
  const double *e;     // [N] e^n (internal order)
  const double *m;     // [N][3] m^n
  const double *le1;   // [N]
  const double *lm1;   // [N][3]
  double *le;          // [N] out
  double *lm;          // [N][3] out
  double *gP, *gJ;     // [N] +=
  double dt, cbar, c, a_rad, r_gas, gamma_gas;
  int newton_max_iter;
};

__device__ double newton_root(double alpha, double beta, double g, int max_iter) {
  double T = g / beta;
  if (alpha > 0.0) T = fmin(T, sqrt(sqrt(g / alpha)));
  bool done = false;
  for (int it = 0; it < max_iter && !done; ++it) {
    const double T2 = T * T;
    const double f = fma(alpha * T2, T2, fma(beta, T, -g));
    const double fp = fma(4.0 * alpha * T2, T, beta);
    const double Tn = T - f / fp;
    if (!(Tn < T)) {
      done = true;
    } else {
      done = (T - Tn <= 1e-15 * T);
      T = Tn;
    }
  }
  return T;
}

// Source adjoint, one warp per cell; intensities, directions and weights in
// the internal (pair-interleaved) angle order.
template <typename R>
__global__ void source_adjoint_kernel(const SrcAdjArgs a, const R *__restrict__ Is,
                                      const R *__restrict__ lI1, R *__restrict__ lIs) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (c >= a.n) return;
  const int lane = threadIdx.x % 32, A = a.A;
  const int kind = a.kind[c];
  const double le1 = a.le1[c];
  const double lm1[3] = {a.lm1[3 * c], a.lm1[3 * c + 1], a.lm1[3 * c + 2]};
  const GasStatic gs = a.gs[c];
  const double rho = gs.rho;
  const double m[3] = {a.m[3 * c], a.m[3 * c + 1], a.m[3 * c + 2]};
  const double cc = a.c, cb = a.cbar, dt = a.dt;
  if (kind == RT_CELL_BOUNDARY) {
    const double2 ax = a.aux[c];
    const double f = (ax.x <= dt) ? 1.0 : dt / ax.x;
    for (int k = lane; k < A; k += 32)
      lIs[(size_t)c * A + k] = R((1.0 - f) * (double)lI1[(size_t)c * A + k]);
    if (lane == 0) {
      a.le[c] = le1;
      for (int d = 0; d < 3; ++d) a.lm[3 * c + d] = lm1[d];
    }
    return;
  }
  const double v[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
  if (kind == RT_CELL_EMITTER) {
    const double2 ax = a.aux[c];
    const double Y = dt * cb * ax.x, isrc = ax.y;
    double lv[3] = {0, 0, 0};
    for (int k = lane; k < A; k += 32) {
      const double *n = a.dir + 3 * k;
      const int q = k;
      const double G = 1.0 - (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / cc;
      const double G4 = G * G * G * G, y = Y * G;
      const double is = (double)Is[(size_t)c * A + q], l1 = (double)lI1[(size_t)c * A + q];
      const double In = ((G4 * is + y * isrc) / (1.0 + y)) / G4;
      lIs[(size_t)c * A + q] = R(l1 / (1.0 + y));
      const double dIdG = (-3.0 * Y * isrc / G4 - Y * In) / (1.0 + y);
      for (int d = 0; d < 3; ++d) lv[d] += -n[d] / cc * dIdG * l1;
    }
    for (int d = 0; d < 3; ++d) lv[d] = warp_sum(lv[d]);
    if (lane == 0) {
      a.le[c] = le1;
      for (int d = 0; d < 3; ++d) a.lm[3 * c + d] = lm1[d] + lv[d] / rho;
    }
    return;
  }
  // ---------------- interior: forward recomputation (as the step, in double)
  const double kP = gs.rkP / rho, kJ = gs.rkJ / rho, kS = gs.rkS / rho;
  double G[kMaxPerLane], wh[kMaxPerLane], It[kMaxPerLane], x[kMaxPerLane], is[kMaxPerLane];
  double Nw = 0.0;
#pragma unroll
  for (int t = 0; t < kMaxPerLane; ++t) {
    const int k = lane + 32 * t;
    G[t] = 1.0;
    wh[t] = It[t] = x[t] = is[t] = 0.0;
    if (k < A) {
      const double *n = a.dir + 3 * k;
      G[t] = 1.0 - (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / cc;
      is[t] = (double)Is[(size_t)c * A + k];
      It[t] = G[t] * G[t] * G[t] * G[t] * is[t];
      wh[t] = a.wt[k] / (G[t] * G[t]);
      x[t] = dt * cb * rho * (kJ + kS) * G[t];
      Nw += wh[t];
    }
  }
  Nw = warp_sum(Nw);
  double SI = 0.0, SG = 0.0;
#pragma unroll
  for (int t = 0; t < kMaxPerLane; ++t) {
    if (lane + 32 * t < A) {
      const double w = wh[t] / Nw;
      SI += w * It[t] / (1.0 + x[t]);
      SG += w * G[t] / (1.0 + x[t]);
    }
  }
  SI = warp_sum(SI);
  SG = warp_sum(SG);
  const double D = 1.0 - dt * cb * rho * kS * SG;
  const double kin = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho;
  const double rcv = rho * a.r_gas / (a.gamma_gas - 1.0);
  const double Tn = (a.e[c] - kin) / rcv;
  const double hJ = 1.0 - dt * cb * rho * kJ * SG / D;
  const double alpha = dt * cc * rho * kP * a.a_rad * hJ;
  const double g = rcv * Tn + dt * cc * rho * 4.0 * kPi * kJ * SI / D;
  const double T = newton_root(alpha, rcv, g, a.newton_max_iter);
  const double B = a.a_rad * T * T * T * T / (4.0 * kPi);
  const double J = (SI + dt * cb * rho * kP * B * SG) / D;
  const double q = dt * cb * rho * (kP * B + kS * J);
  // ---------------- reverse
  const double ldE = cc / cb * le1;
  const double ldF[3] = {lm1[0] / (cc * cb), lm1[1] / (cc * cb), lm1[2] / (cc * cb)};
  double lG[kMaxPerLane], lIt[kMaxPerLane], lx[kMaxPerLane], lIsv[kMaxPerLane];
  double lq = 0.0;
#pragma unroll
  for (int t = 0; t < kMaxPerLane; ++t) {
    const int k = lane + 32 * t;
    lG[t] = lIt[t] = lx[t] = lIsv[t] = 0.0;
    if (k < A) {
      const double *n = a.dir + 3 * k;
      const double ex =
          4.0 * kPi * a.wt[k] * (ldE + cc * (n[0] * ldF[0] + n[1] * ldF[1] + n[2] * ldF[2]));
      lIsv[t] = ex;
      const double lIn = (double)lI1[(size_t)c * A + k] - ex;
      const double G4 = G[t] * G[t] * G[t] * G[t];
      const double Itn = (It[t] + q * G[t]) / (1.0 + x[t]);
      const double In = Itn / G4;
      const double lItn = lIn / G4;
      lG[t] = -4.0 * In / G[t] * lIn + q * lItn / (1.0 + x[t]);
      lIt[t] = lItn / (1.0 + x[t]);
      lq += G[t] * lItn / (1.0 + x[t]);
      lx[t] = -Itn * lItn / (1.0 + x[t]);
    }
  }
  lq = warp_sum(lq);
  double gP = dt * cb * rho * B * lq, gJ = 0.0;
  double lB = dt * cb * rho * kP * lq;
  const double lJ = dt * cb * rho * kS * lq;
  double lSI = lJ / D;
  double lSG = dt * cb * rho * kP * B * lJ / D;
  double lD = -J * lJ / D;
  lB += dt * cb * rho * kP * SG * lJ / D;
  gP += dt * cb * rho * B * SG * lJ / D;
  const double lT = a.a_rad * T * T * T / kPi * lB;
  const double Fp = 4.0 * alpha * T * T * T + rcv;
  const double lalpha = -T * T * T * T / Fp * lT;
  const double lg = lT / Fp;
  const double lTn = rcv * lg;
  lSI += dt * cc * rho * 4.0 * kPi * kJ / D * lg;
  lD += -dt * cc * rho * 4.0 * kPi * kJ * SI / (D * D) * lg;
  gJ += dt * cc * rho * 4.0 * kPi * SI / D * lg;
  gP += dt * cc * rho * a.a_rad * hJ * lalpha;
  gJ += dt * cc * rho * kP * a.a_rad * (-dt * cb * rho * SG / D) * lalpha;
  lSG += dt * cc * rho * kP * a.a_rad * (-dt * cb * rho * kJ / D) * lalpha;
  lD += dt * cc * rho * kP * a.a_rad * (dt * cb * rho * kJ * SG / (D * D)) * lalpha;
  const double le_out = le1 + lTn / rcv;
  const double lkin = -lTn / rcv;
  lSG += -dt * cb * rho * kS * lD;
  double lwt[kMaxPerLane];
  double swl = 0.0;
#pragma unroll
  for (int t = 0; t < kMaxPerLane; ++t) {
    lwt[t] = 0.0;
    if (lane + 32 * t < A) {
      const double w = wh[t] / Nw;
      const double r = 1.0 / (1.0 + x[t]);
      lwt[t] = (It[t] * lSI + G[t] * lSG) * r;
      lIt[t] += w * lSI * r;
      lG[t] += w * lSG * r;
      lx[t] += -w * (It[t] * lSI + G[t] * lSG) * r * r;
      swl += w * lwt[t];
    }
  }
  swl = warp_sum(swl);
  double lv[3] = {0.0, 0.0, 0.0};
  double gJx = 0.0;
#pragma unroll
  for (int t = 0; t < kMaxPerLane; ++t) {
    const int k = lane + 32 * t;
    if (k < A) {
      gJx += dt * cb * rho * G[t] * lx[t];
      lG[t] += dt * cb * rho * (kJ + kS) * lx[t];
      const double lwh = (lwt[t] - swl) / Nw;
      lG[t] += -2.0 * wh[t] / G[t] * lwh;
      lIsv[t] += G[t] * G[t] * G[t] * G[t] * lIt[t];
      lG[t] += 4.0 * G[t] * G[t] * G[t] * is[t] * lIt[t];
      const double *n = a.dir + 3 * k;
      for (int d = 0; d < 3; ++d) lv[d] += -n[d] / cc * lG[t];
      lIs[(size_t)c * A + k] = R(lIsv[t]);
    }
  }
  gJx = warp_sum(gJx);
  for (int d = 0; d < 3; ++d) lv[d] = warp_sum(lv[d]);
  if (lane == 0) {
    a.le[c] = le_out;
    for (int d = 0; d < 3; ++d) a.lm[3 * c + d] = lm1[d] + m[d] / rho * lkin + lv[d] / rho;
    a.gP[c] += gP;
    a.gJ[c] += gJ + gJx;
  }
}

unsigned rows_grid(int64_t n) { return (unsigned)((n + kThreads / 32 - 1) / (kThreads / 32)); }

// caller order -> internal order for per-cell vectors of width w (double)
__global__ void gather_cells(const double *__restrict__ src, double *__restrict__ dst,
                             const int64_t *__restrict__ cell_of, int64_t n, int w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < w; ++k) dst[(size_t)i * w + k] = src[(size_t)cell_of[i] * w + k];
}
// internal order -> caller order; accumulate when add != 0
__global__ void scatter_cells(const double *__restrict__ src, double *__restrict__ dst,
                              const int64_t *__restrict__ cell_of, int64_t n, int w, int add) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < w; ++k) {
    double *p = dst + (size_t)cell_of[i] * w + k;
    *p = add ? *p + src[(size_t)i * w + k] : src[(size_t)i * w + k];
  }
}

template <typename R> cudaError_t run_adjoint(rt_state *s, const R *I_int, const R *lI1_int,
                                              R *lI_int, double dt, double *ws) {
  const int64_t N = s->n_cells;
  const int A = s->n_angles;
  R *Is = reinterpret_cast<R *>(s->d_adj[0]);
  R *lIs = reinterpret_cast<R *>(s->d_adj[1]);
  const auto *slot = reinterpret_cast<const typename SlotOf<R>::type *>(s->d_slot);
  const R *iv = reinterpret_cast<const R *>(s->d_inv_vol);
  const R *dir = reinterpret_cast<const R *>(s->d_dir);
  transport_kernel<R><<<rows_grid(N), kThreads, 0, s->stream>>>(s->d_ptr, s->d_nbr, slot, s->d_wface,
                                                                 iv, dir, I_int, Is, N, A, s->quad_end,
                                                                 R(dt));
  SrcAdjArgs a;
  a.n = N;
  a.A = A;
  a.gs = s->d_gs;
  a.kind = s->d_kind;
  a.aux = s->d_aux;
  a.dir = s->d_dir64;
  a.wt = s->d_wt64;
  a.e = ws;
  a.m = ws + N;
  a.le1 = ws + 4 * N;
  a.lm1 = ws + 5 * N;
  a.le = ws + 8 * N;
  a.lm = ws + 9 * N;
  a.gP = ws + 12 * N;
  a.gJ = ws + 13 * N;
  a.dt = dt;
  a.cbar = s->params.cbar;
  a.c = s->params.c;
  a.a_rad = s->params.a_rad;
  a.r_gas = s->params.r_gas;
  a.gamma_gas = s->params.gamma_gas;
  a.newton_max_iter = s->params.newton_max_iter;
  source_adjoint_kernel<R><<<rows_grid(N), kThreads, 0, s->stream>>>(a, Is, lI1_int, lIs);
  transport_adjoint_kernel<R><<<rows_grid(N), kThreads, 0, s->stream>>>(
      s->d_ptr, s->d_nbr, slot, s->d_wface, iv, dir, lIs, lI_int, N, A, s->quad_end, R(dt));
  s->launches += 3;
  return cudaGetLastError();
}

}  // namespace

cudaError_t adjoint_step(rt_state *s, double dt, const void *I, const double *e, const double *m,
                         const void *lI1, const double *le1, const double *lm1, void *lI,
                         double *le, double *lm, double *gP, double *gJ) {
  // all pointers are device pointers in the caller's order; the internal
  // copies use dense rows (stride A)
  const int64_t N = s->n_cells;
  const unsigned g1 = (unsigned)((N + kThreads - 1) / kThreads);
  double *ws = s->d_adj_ws;  // [14 N]: e, m, (pad), le1, lm1, le, lm, gP, gJ (internal)
  void *I_int = s->d_adj[2], *lI1_int = s->d_adj[3], *lI_int = s->d_adj[4];
  cudaError_t err = launch_permute_in(s, I, I_int, s->n_angles);
  if (err == cudaSuccess) err = launch_permute_in(s, lI1, lI1_int, s->n_angles);
  if (err != cudaSuccess) return err;
  gather_cells<<<g1, kThreads, 0, s->stream>>>(e, ws, s->d_cell_of, N, 1);
  gather_cells<<<g1, kThreads, 0, s->stream>>>(m, ws + N, s->d_cell_of, N, 3);
  gather_cells<<<g1, kThreads, 0, s->stream>>>(le1, ws + 4 * N, s->d_cell_of, N, 1);
  gather_cells<<<g1, kThreads, 0, s->stream>>>(lm1, ws + 5 * N, s->d_cell_of, N, 3);
  err = cudaMemsetAsync(ws + 12 * N, 0, sizeof(double) * 2 * N, s->stream);
  if (err != cudaSuccess) return err;
  s->launches += 4;
  if (s->precision == RT_FP32)
    err = run_adjoint<float>(s, (const float *)I_int, (const float *)lI1_int, (float *)lI_int, dt,
                             ws);
  else
    err = run_adjoint<double>(s, (const double *)I_int, (const double *)lI1_int,
                              (double *)lI_int, dt, ws);
  if (err != cudaSuccess) return err;
  err = launch_permute_out(s, lI_int, lI, s->n_angles);
  if (err != cudaSuccess) return err;
  scatter_cells<<<g1, kThreads, 0, s->stream>>>(ws + 8 * N, le, s->d_cell_of, N, 1, 0);
  scatter_cells<<<g1, kThreads, 0, s->stream>>>(ws + 9 * N, lm, s->d_cell_of, N, 3, 0);
  scatter_cells<<<g1, kThreads, 0, s->stream>>>(ws + 12 * N, gP, s->d_cell_of, N, 1, 1);
  scatter_cells<<<g1, kThreads, 0, s->stream>>>(ws + 13 * N, gJ, s->d_cell_of, N, 1, 1);
  s->launches += 4;
  return cudaGetLastError();
}

}  // namespace rt
