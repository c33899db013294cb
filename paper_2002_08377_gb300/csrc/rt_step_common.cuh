// Device helpers of the step kernel (rt_step.cu).
#pragma once

#include <cuda_runtime.h>

#include "rt_internal.cuh"

namespace rt {
namespace step {

constexpr int KT = 8;         // threads per cell
constexpr int NT = KT * CPB;  // threads per block

// ------------------------------------------------------------ pair arithmetic
template <typename R> struct P2;
template <> struct P2<float> { using t = float2; };
template <> struct P2<double> { using t = double2; };
template <typename R> using pair_t = typename P2<R>::t;

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) {
  return make_double2(a.x * b.x, a.y * b.y);
}
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 padd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}

__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ double2 psub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}

// Reciprocal.  Float: the PTX approximate reciprocal (one MUFU operation,
// relative error below 2^-22, inside the float state's error budget; the
// arguments are Gamma^k (1 + x Gamma) and 1 + dt cbar rho kappa S_G, normal
// floats, so flushing subnormals changes nothing).  Double: that estimate
// refined by two Newton steps r <- r (2 - x r) (about 1 ulp) where x and
// 1/x are normal floats (|x| in [2^-125, 2^126)); any other x (physical
// units make dt/V or cbar A far from 1) takes the IEEE double division.
__device__ __forceinline__ float rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double rcp(double x) {
  // |x| in [2^-125, 2^126) <=> biased exponent in [898, 1149), tested on the
  // integer pipe (the FP64 pipe is the double kernels' bottleneck)
  const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
  if (ex - 898u >= 251u) return 1.0 / x;
  double r = (double)rcp((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}
template <typename R> __device__ __forceinline__ pair_t<R> prcp(pair_t<R> v) {
  return mk(rcp(v.x), rcp(v.y));
}

// Four consecutive reals (16-byte aligned for float, 32 for double).
__device__ __forceinline__ void store4(float *p, float x, float y, float z, float w) {
  *reinterpret_cast<float4 *>(p) = make_float4(x, y, z, w);
}
__device__ __forceinline__ void store4(double *p, double x, double y, double z, double w) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(x, y);
  reinterpret_cast<double2 *>(p)[1] = make_double2(z, w);
}

// Direction (x, y, z) of pair p from the [A][4] direction table.
__device__ __forceinline__ void load_dir(const float *dir, int p, float &x, float &y, float &z) {
  const float4 t = __ldg(reinterpret_cast<const float4 *>(dir) + p);
  x = t.x;
  y = t.y;
  z = t.z;
}
__device__ __forceinline__ void load_dir(const double *dir, int p, double &x, double &y,
                                         double &z) {
  const double2 t = __ldg(reinterpret_cast<const double2 *>(dir) + 2 * p);
  x = t.x;
  y = t.y;
  z = __ldg(dir + 4 * p + 2);
}

template <typename R> __device__ __forceinline__ typename SlotOf<R>::type load_slot(
    const typename SlotOf<R>::type *p);
template <> __device__ __forceinline__ SlotF load_slot<float>(const SlotF *p) {
  float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  return {v.x, v.y, v.z, v.w};
}
template <> __device__ __forceinline__ SlotD load_slot<double>(const SlotD *p) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  return {a.x, a.y, b.x, b.y};
}

// n_a . s of a slot (float) or cbar A ((n_ax n_fx + n_ay n_fy) + n_az n_fz)
// without contraction (double); and the slot's A w . n
__device__ __forceinline__ float slot_dot(float x, float y, float z, const SlotF &s) {
  return fmaf(x, s.sx, fmaf(y, s.sy, z * s.sz));
}
__device__ __forceinline__ double slot_dot(double x, double y, double z, const SlotD &s) {
  return __dmul_rn(s.ca, __dadd_rn(__dadd_rn(__dmul_rn(x, s.nx), __dmul_rn(y, s.ny)),
                                   __dmul_rn(z, s.nz)));
}
__device__ __forceinline__ float slot_w(const SlotF &s, const double *, int64_t) { return s.w; }
__device__ __forceinline__ double slot_w(const SlotD &, const double *wf, int64_t k) {
  return wf[k];
}

template <typename T> __device__ __forceinline__ T cell_sum(T v) {
#pragma unroll
  for (int o = KT / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned cell_or(unsigned v) {
#pragma unroll
  for (int o = KT / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Positive root of alpha T^4 + beta T = g (alpha >= 0, beta > 0, g >= 0).
// f is increasing and convex on T >= 0, so one Newton step from any T0 >= 0
// lands at or above the root, and Newton from there decreases monotonically
// onto it.  T0 is the gas temperature before the step (close to the root
// when the step changes it little); the first iterate is capped by the
// bound g / beta.  The iteration stops when an iterate fails to decrease or
// moves by at most `tol` of itself.  Returns 1 if it did not converge.
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }

template <typename T_>
__device__ __forceinline__ int quartic_root(T_ alpha, T_ beta, T_ g, T_ T0, T_ tol, int max_iter,
                                            T_ *T_out) {
  T_ T = T0 > T_(0) ? T0 : T_(0);
  {
    const T_ T2 = T * T;
    const T_ f = fma(alpha * T2, T2, fma(beta, T, -g));
    const T_ fp = fma(T_(4) * alpha * T2, T, beta);
    T = fmin(T - qdiv(f, fp), qdiv(g, beta));
  }
  bool done = false;
  for (int it = 0; it < max_iter && !done; ++it) {
    const T_ T2 = T * T;
    const T_ f = fma(alpha * T2, T2, fma(beta, T, -g));
    const T_ fp = fma(T_(4) * alpha * T2, T, beta);
    const T_ Tn = T - qdiv(f, fp);
    if (!(Tn < T)) {
      done = true;
    } else {
      done = (T - Tn <= tol * T);
      T = Tn;
    }
  }
  *T_out = T;
  return done ? 0 : 1;
}

// One Newton step in double on alpha T^k + beta T = g (k = 4 + beta_P) from
// the float root T0 of the float coefficients alpha, g: the residual f in
// double, f' and the quotient f / f' in float.  From a float-accurate start
// (relative error e0 of a few float ulp, ~1e-7) the step leaves about
// e0 (float epsilon + e0), ~1e-13, below the float rounding of the q it
// feeds.  beta_P_f == 0 selects the quartic (T^3 by multiplication); f' in
// float costs nothing in accuracy since the quotient is taken in float.
__device__ __forceinline__ double refine_root(float alpha, float beta_P_f, double beta_P,
                                              double beta, float g, float T0) {
  const double T = (double)T0;
  double Tk1;
  float kf;
  if (beta_P_f == 0.0f) {
    Tk1 = (T * T) * T;
    kf = 4.0f;
  } else {
    Tk1 = pow(T, 3.0 + beta_P);
    kf = 4.0f + beta_P_f;
  }
  const double f = fma((double)alpha * Tk1, T, fma(beta, T, -(double)g));
  const float fp = fmaf(kf * alpha, (float)Tk1, (float)beta);
  return T - (double)((float)f * rcp(fp));
}

// Positive root of alpha T^k + beta T = g for k >= 1 (alpha >= 0, beta > 0,
// g >= 0): the temperature equation when kappa_P is proportional to T^(k-4).
// The left side is increasing and convex for T >= 0, so, as for
// quartic_root, one Newton step from T0 >= 0 lands at or above the root
// (capped by g / beta) and the iterates then decrease monotonically onto it.
// Returns 1 if it did not converge.
__device__ __forceinline__ float ppow(float x, float k) { return powf(x, k); }
__device__ __forceinline__ double ppow(double x, double k) { return pow(x, k); }
template <typename T_>
__device__ int power_root(T_ alpha, T_ k, T_ beta, T_ g, T_ T0, T_ tol, int max_iter, T_ *T_out) {
  T_ T = T0 > T_(0) ? T0 : T_(0);
  {
    const T_ Tk1 = ppow(T, k - T_(1));
    const T_ f = fma(alpha * Tk1, T, fma(beta, T, -g));
    const T_ fp = fma(k * alpha, Tk1, beta);
    T = fmin(T - qdiv(f, fp), qdiv(g, beta));
  }
  bool done = false;
  for (int it = 0; it < max_iter && !done; ++it) {
    const T_ Tk1 = ppow(T, k - T_(1));
    const T_ f = fma(alpha * Tk1, T, fma(beta, T, -g));
    const T_ fp = fma(k * alpha, Tk1, beta);
    const T_ Tn = T - qdiv(f, fp);
    if (!(Tn < T)) {
      done = true;
    } else {
      done = (T - Tn <= tol * T);
      T = Tn;
    }
  }
  *T_out = T;
  return done ? 0 : 1;
}

// u > 0, the upwind test.  Double: from the sign and high word of u, on the
// integer pipe (differs from u > 0 only for |u| below 2^-1042, whose flux is
// far below rounding).
__device__ __forceinline__ bool positive(float u) { return u > 0.0f; }
__device__ __forceinline__ bool positive(double u) { return __double2hiint(u) > 0; }

// One face's contribution to sum_f u I_up for one of the thread's pairs:
// (vx, vy) the neighbour's (I_p, I_{p+H}), Ia / Ib the cell's own values.
template <typename R, bool MOVING>
__device__ __forceinline__ void face_pair(R d, R w, R vx, R vy, R Ia, R Ib, R &acca, R &accb) {
  if (MOVING) {
    const R ua = d - w, ub = -d - w;
    acca = fma(ua, positive(ua) ? Ia : vx, acca);
    accb = fma(ub, positive(ub) ? Ib : vy, accb);
  } else {
    // u_a = d, u_b = -d: exactly one of the pair takes the neighbour's value
    const bool out = positive(d);
    acca = fma(d, out ? Ia : vx, acca);
    accb = fma(-d, out ? vy : Ib, accb);
  }
}

}  // namespace step
}  // namespace rt
