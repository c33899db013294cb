// Fused radiation step: upwind transport (Sec. 3.2) + implicit comoving
// source update with gas exchange (Sec. 3.3), boundary cells (Sec. 3.5) and
// emitter cells (Sec. 3.6), one kernel per step.
//
// Layout: the intensity row of a cell stores the A/2 antipodal pairs
// (angle p, angle p + A/2) side by side, so one 8-byte (float) or 16-byte
// (double) load fetches a pair.  The flux coefficient of the antipode through
// a face is u(p + A/2) = -(n_p . s) - w, so one dot product serves both
// angles; on a static mesh exactly one of the two is inflow.
//
// Block = 32 cells x 8 threads; thread `sub` of a cell owns the pairs
// p = sub + 8 j (j < PPT).  Registers are capped so that four blocks share an
// SM: the step is latency-bound, and resident warps matter more than the
// shared-memory staging of neighbour rows that an earlier variant used.
// Phases (separated by __syncthreads):
//   A  all threads: transport over the cell's faces in slot order (no
//      atomics, deterministic), comoving weights and the angular sums of
//      Eq. (Jcom); each cell's 8 lanes reduce with shuffles;
//   B  warp 0, one lane per cell: the gas temperature quartic in double
//      (float states: float Newton plus one double Newton step);
//   C  all threads: new intensities, store, radiation change per cell;
//   D  warp 0, one lane per cell: gas energy / momentum (or tally) update in
//      double (Eqs. gas1, gas2).
// The double-precision work is lane-per-cell because GB300's FP64 rate is a
// small fraction of its FP32 rate.  Float states use the packed f32x2 FMA.
#include <cuda_runtime.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

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

// Reciprocal: float uses the hardware approximation (relative error ~1e-7,
// inside the float state's error budget); double refines the float estimate
// with two Newton steps (about 1 ulp).  Arguments are 1 + x (x >= 0) and
// Gamma^2, far inside float range.
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp(double x) {
  double r = (double)__fdividef(1.0f, (float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
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
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Positive root of alpha T^4 + beta T = g (alpha >= 0, beta > 0, g >= 0).
// f is increasing and convex on T > 0, so Newton from any point at or above
// the root decreases monotonically onto it.  Double states: start at
// min(g/beta, (g/alpha)^(1/4)) and stop when an iterate fails to decrease or
// moves by at most 1e-15 of itself.  Float states: the same iteration in
// float to a relative 1e-7, then one Newton step in double (the float
// root's error ~1e-7 becomes ~1e-14); coefficients outside float range fall
// back to the double iteration.  Returns 1 if it did not converge.
__device__ __forceinline__ float fp_of(float af, float bf, float t) {
  return fmaf(4.0f * af * t * t, t, bf);
}

template <bool FLOAT_STATE>
__device__ __forceinline__ int quartic_root(double alpha, double beta, double g, int max_iter,
                                            double *T_out) {
  if (FLOAT_STATE) {
    const float af = (float)alpha, bf = (float)beta, gf = (float)g;
    float t = __fdividef(gf, bf);
    if (af > 0.0f) t = fminf(t, sqrtf(sqrtf(__fdividef(gf, af))));
    bool done = false;
    for (int it = 0; it < max_iter && !done; ++it) {
      const float t2 = t * t;
      const float f = fmaf(af * t2, t2, fmaf(bf, t, -gf));
      const float fp = fmaf(4.0f * af * t2, t, bf);
      const float tn = t - __fdividef(f, fp);
      if (!(tn < t)) {
        done = true;
      } else {
        done = (t - tn <= 1e-7f * t);
        t = tn;
      }
    }
    if (isfinite(t) && t >= 0.0f && isfinite(fp_of(af, bf, t))) {
      if (!done) {
        *T_out = t;
        return 1;
      }
      const double T = t, T2 = T * T;
      const double f = fma(alpha * T2, T2, fma(beta, T, -g));
      const double fp = fma(4.0 * alpha * T2, T, beta);
      *T_out = fma(-f, rcp(fp), T);
      return 0;
    }
  }
  double T = g / beta;
  if (alpha > 0.0) T = fmin(T, sqrt(sqrt(g / alpha)));
  bool done = false;
  int it = 0;
  while (!done && it < max_iter) {
    const double T2 = T * T;
    const double f = fma(alpha * T2, T2, fma(beta, T, -g));
    const double fp = fma(4.0 * alpha * T2, T, beta);
    const double Tn = T - f / fp;
    ++it;
    if (!(Tn < T)) {
      done = true;
    } else {
      done = (T - Tn <= 1e-15 * T);
      T = Tn;
    }
  }
  *T_out = T;
  return done ? 0 : 1;
}

template <typename R> struct Shared {
  GasStatic gs[CPB];  // gas of the block's cells, prefetched for warp 0
  GasDyn gd[CPB];
  R sI[CPB], sG[CPB], s1[CPB];  // the sums of Eq. (Jcom) and sum w~/(1+x), unnormalised
  R q[CPB];                     // dt cbar rho (kP B + kS J) per interior cell
  R dE[CPB], dF[3][CPB];        // sum w (I* - I') and sum w n (I* - I')
  unsigned bad[CPB];
};

// One face's contribution to sum_f u I_up for the thread's pairs: v is the
// neighbour's (I_p, I_{p+H}) pair, Ia/Ib the cell's own values.
template <typename R, bool MOVING>
__device__ __forceinline__ void face_pair(R d, R w, pair_t<R> v, R Ia, R Ib, R &acca, R &accb) {
  if (MOVING) {
    const R ua = d - w, ub = -d - w;
    acca = fma(ua, ua > R(0) ? Ia : v.x, acca);
    accb = fma(ub, ub > R(0) ? Ib : v.y, accb);
  } else {
    // u_a = d, u_b = -d: exactly one of the pair takes the neighbour's value
    const bool out = d > R(0);
    acca = fma(d, out ? Ia : v.x, acca);
    accb = fma(-d, out ? v.y : Ib, accb);
  }
}

// sum_f u I_up over the slots [k0, k1) of one cell, neighbour rows read
// through nbr[k] (L1/L2 serve the reuse between neighbouring cells; cells are
// in Morton order).  FULL: every lane owns exactly PPT pairs (A/2 divisible
// by the threads per cell).
template <typename R, int PPT, bool MOVING, bool FULL, typename S>
__device__ __forceinline__ void face_sum(const S *__restrict__ slot, const int32_t *__restrict__ nbr,
                                         const double *__restrict__ wface, int64_t k0, int64_t k1,
                                         const R *__restrict__ I_in, int A, int sub,
                                         const R (&nx)[PPT], const R (&ny)[PPT],
                                         const R (&nz)[PPT], const R (&Ia)[PPT], const R (&Ib)[PPT],
                                         R (&acca)[PPT], R (&accb)[PPT], int np) {
  using V = pair_t<R>;
#pragma unroll 2
  for (int64_t k = k0; k < k1; ++k) {
    const S s = slot[k];
    const V *In = reinterpret_cast<const V *>(I_in + (size_t)nbr[k] * A) + sub;
    const R w = MOVING ? slot_w(s, wface, k) : R(0);
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      if (FULL || j < np) {
        const V v = In[KT * j];
        face_pair<R, MOVING>(slot_dot(nx[j], ny[j], nz[j], s), w, v, Ia[j], Ib[j], acca[j],
                             accb[j]);
      }
    }
  }
}

template <typename R, int PPT, bool MOVING, bool FULL>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 4 : 2) step_kernel(const StepArgs<R> a) {
  using V = pair_t<R>;
  using S = typename SlotOf<R>::type;
  __shared__ Shared<R> sh;
  const int lc = threadIdx.x / KT;
  const int sub = threadIdx.x % KT;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t cell = (int64_t)blockIdx.x * CPB + lc;
  const bool live = cell < a.n_cells;
  const int64_t c = live ? cell : a.n_cells - 1;  // dead lanes shadow the last cell
  const int A = a.n_angles, H = a.half;
  const int np = FULL ? PPT : (H - sub + KT - 1) / KT;  // pairs p = sub + KT j < H

  // warp 0 prefetches its cells' gas state for phases B and D
  const int64_t cl = (int64_t)blockIdx.x * CPB + lane;  // warp 0: lane-per-cell
  if (warp == 0 && lane < CPB && cl < a.n_cells) {
    const char *g = reinterpret_cast<const char *>(a.gs + cl);
    const char *d = reinterpret_cast<const char *>(a.gd + cl);
#pragma unroll
    for (int k = 0; k < 4; ++k) cp_async16(reinterpret_cast<char *>(&sh.gs[lane]) + 16 * k, g + 16 * k);
#pragma unroll
    for (int k = 0; k < 2; ++k) cp_async16(reinterpret_cast<char *>(&sh.gd[lane]) + 16 * k, d + 16 * k);
  }

  // ---------------- phase A: transport, I* = I - dt/V sum_f u I_up
  R nx[PPT], ny[PPT], nz[PPT], Ia[PPT], Ib[PPT], acca[PPT], accb[PPT];
  {
    const V *Ic = reinterpret_cast<const V *>(a.I_in + (size_t)c * A) + sub;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const bool v = FULL || j < np;
      const int p = v ? sub + KT * j : 0;
      nx[j] = a.dir[4 * p];
      ny[j] = a.dir[4 * p + 1];
      nz[j] = a.dir[4 * p + 2];
      const V t = v ? Ic[KT * j] : mk(R(0), R(0));
      Ia[j] = t.x;
      Ib[j] = t.y;
      acca[j] = R(0);
      accb[j] = R(0);
    }
  }
  face_sum<R, PPT, MOVING, FULL>(a.slot, a.nbr, a.wface, a.ptr[c], a.ptr[c + 1], a.I_in, A, sub, nx,
                                 ny, nz, Ia, Ib, acca, accb, np);
  {
    const R dtv = a.dt_r * a.inv_vol[c];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      Ia[j] = fma(-dtv, acca[j], Ia[j]);  // I*
      Ib[j] = fma(-dtv, accb[j], Ib[j]);
    }
  }

  // comoving frame (first order in v/c): Gamma = 1 -+ v.n / c, and the
  // angular sums of Eq. (Jcom): w~ = w / Gamma^2 (normalised by their sum),
  // S_I = sum w~ Gamma^4 I* / (1 + x Gamma), S_G = sum w~ Gamma / (1 + x Gamma)
  const int kind = a.kind[c];
  const R icr = a.inv_c_r;
  const R vxc = a.cellv[4 * c] * icr, vyc = a.cellv[4 * c + 1] * icr,
          vzc = a.cellv[4 * c + 2] * icr;
  const R xs = a.dt_cbar_r * a.cellv[4 * c + 3];
  const V *W2 = reinterpret_cast<const V *>(a.wt2) + sub;  // (w_p, w_{p+H})
  R Ga[PPT];
  R sI = 0, sG = 0, s1 = 0;  // unnormalised: the normalisation cancels in phase B
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    Ga[j] = R(1) - fma(vxc, nx[j], fma(vyc, ny[j], vzc * nz[j]));
    if (FULL || j < np) {
      const R ga = Ga[j], gb = R(2) - ga;
      const R ga2 = ga * ga, gb2 = gb * gb;
      const V w = W2[KT * j];
      const R wca = w.x * rcp(ga2), wcb = w.y * rcp(gb2);
      const R ta = wca * rcp(fma(xs, ga, R(1))), tb = wcb * rcp(fma(xs, gb, R(1)));
      s1 += ta + tb;
      sI = fma(ta, ga2 * ga2 * Ia[j], fma(tb, gb2 * gb2 * Ib[j], sI));
      sG = fma(ta, ga, fma(tb, gb, sG));
    }
  }
  sI = cell_sum(sI);
  sG = cell_sum(sG);
  s1 = cell_sum(s1);
  if (sub == 0) {
    sh.sI[lc] = sI;
    sh.sG[lc] = sG;
    sh.s1[lc] = s1;
  }
  if (warp == 0) cp_async_wait_all();
  __syncthreads();

  // ---------------- phase B: temperature quartic, one lane per cell
  if (warp == 0 && lane < CPB) {
    R q = 0;
    unsigned bad = 0;
    if (cl < a.n_cells && a.kind[cl] == RT_CELL_INTERIOR) {
      // With w~ normalised, x_a = dt cbar rho (kJ + kS) Gamma_a and the sums
      // S_I, S_G of Eq. (Jcom), S_1 = sum w~ / (1 + x):
      //   D = 1 - dt cbar rho kS S_G = S_1 + dt cbar rho kJ S_G,
      //   1 - dt cbar rho kJ S_G / D = S_1 / D,
      // so the quartic alpha T^4 + rho c_v T = g of Eq. (com rad thermal disc)
      // has alpha = dt c a rho kP S_1 / D and g = (e - kinetic) +
      // dt c 4 pi rho kJ S_I / D: sums of positive terms, no cancellation when
      // x >> 1.  The weight normalisation cancels in every ratio.
      const GasStatic g = sh.gs[lane];
      const GasDyn d = sh.gd[lane];
      const double SI = (double)sh.sI[lane], SG = (double)sh.sG[lane], S1 = (double)sh.s1[lane];
      const double dJ = a.k_dcr * g.rkJ, dP = a.k_dcr * g.rkP, dS = a.k_dcr * g.rkS;
      const double rU = rcp(fma(dJ, SG, S1));
      const double kin = 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * g.inv_rho;
      const double alpha = a.k_alpha * g.rkP * S1 * rU;
      const double gq = (d.e - kin) + a.k_g * g.rkJ * SI * rU;
      double T = 0.0;
      if (!(gq >= 0.0) || !(alpha >= 0.0)) {
        bad |= ST_NONFINITE;
      } else if (quartic_root<sizeof(R) == 4>(alpha, g.rcv, gq, a.newton_max_iter, &T)) {
        bad |= ST_NONCONV;
      }
      const double B = a.a_rad * (T * T) * (T * T) * (1.0 / (4.0 * kPi));
      const double J = fma(dP * B, SG, SI) * rU;  // the J~ of Eq. (Jcom)
      q = R(fma(dP, B, dS * J));
    }
    sh.q[lane] = q;
    sh.bad[lane] = bad;
  }
  __syncthreads();

  // ---------------- phase C: new intensities and the radiation change
  R de = 0, dfx = 0, dfy = 0, dfz = 0;
  unsigned nonfinite = 0;
  {
    // boundary: I' = I* - (I* - I0) f; interior: I~' = (I~ + q Gamma) / (1 + x Gamma),
    // i.e. I' = (I* + q / Gamma^3) / (1 + x Gamma); emitter: the same with
    // x -> dt cbar (rho kappa)_src and q -> that rate times I_src (Sec. 3.6)
    R f = 0, qq = 0, xx = xs;
    const V *I0 = nullptr;
    if (kind == RT_CELL_BOUNDARY) {
      const double2 ax = a.aux[c];
      f = R((ax.x <= a.dt) ? 1.0 : a.dt / ax.x);
      I0 = reinterpret_cast<const V *>(a.I0 + (size_t)a.bc_row[c] * A) + sub;
    } else if (kind == RT_CELL_EMITTER) {
      const double2 ax = a.aux[c];
      xx = R(a.dt * a.cbar * ax.x);
      qq = xx * R(ax.y);
    } else {
      qq = sh.q[lc];
    }
    V *Io = reinterpret_cast<V *>(a.I_out + (size_t)c * A) + sub;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      if (FULL || j < np) {
        R na, nb;
        if (kind == RT_CELL_BOUNDARY) {
          const V t = I0[KT * j];
          na = fma(-f, Ia[j] - t.x, Ia[j]);
          nb = fma(-f, Ib[j] - t.y, Ib[j]);
        } else {
          const R ga = Ga[j], gb = R(2) - ga;
          const R ra = rcp(ga * ga * ga), rb = rcp(gb * gb * gb);
          na = fma(qq, ra, Ia[j]) * rcp(fma(xx, ga, R(1)));
          nb = fma(qq, rb, Ib[j]) * rcp(fma(xx, gb, R(1)));
        }
        if (live) Io[KT * j] = mk(na, nb);
        if (!isfinite(na) || !isfinite(nb)) nonfinite = ST_NONFINITE;
        const V w = W2[KT * j];
        const R da = w.x * (Ia[j] - na), db = w.y * (Ib[j] - nb);
        de += da + db;
        const R df = da - db;  // the antipode has direction -n
        dfx = fma(nx[j], df, dfx);
        dfy = fma(ny[j], df, dfy);
        dfz = fma(nz[j], df, dfz);
      }
    }
  }
  de = cell_sum(de);
  dfx = cell_sum(dfx);
  dfy = cell_sum(dfy);
  dfz = cell_sum(dfz);
  nonfinite = cell_or(nonfinite);
  if (sub == 0) {
    sh.dE[lc] = de;
    sh.dF[0][lc] = dfx;
    sh.dF[1][lc] = dfy;
    sh.dF[2][lc] = dfz;
    sh.bad[lc] |= nonfinite;
  }
  __syncthreads();

  // ---------------- phase D: gas exchange (Eqs. gas1, gas2), one lane per cell
  if (warp == 0 && lane < CPB && cl < a.n_cells) {
    // dE_gas = (c/cbar) 4 pi sum w dI, d(rho v) = (4 pi c sum w n dI) / (c cbar)
    const double dE = a.k_fe * (double)sh.dE[lane];
    const double dx = a.k_fm * (double)sh.dF[0][lane], dy = a.k_fm * (double)sh.dF[1][lane],
                 dz = a.k_fm * (double)sh.dF[2][lane];
    if (a.kind[cl] == RT_CELL_INTERIOR) {
      GasDyn d = sh.gd[lane];
      d.e += dE;
      d.mx += dx;
      d.my += dy;
      d.mz += dz;
      a.gd[cl] = d;
      const double ir = sh.gs[lane].inv_rho;  // frame velocity of the next step
      a.cellv[4 * cl] = R(d.mx * ir);
      a.cellv[4 * cl + 1] = R(d.my * ir);
      a.cellv[4 * cl + 2] = R(d.mz * ir);
    } else {
      double *x = a.ext + 4 * cl;
      x[0] += dE;
      x[1] += dx;
      x[2] += dy;
      x[3] += dz;
    }
    const unsigned bad = sh.bad[lane];
    if (bad) {
      atomicOr(a.status, bad);
      atomicMin(a.bad_cell, (unsigned long long)cl);
    }
  }
}

template <typename R, int PPT, bool MOVING, bool FULL>
cudaError_t launch_t(rt_state *s, double dt) {
  StepArgs<R> a;
  a.n_cells = s->n_cells;
  a.n_angles = s->n_angles;
  a.half = s->n_angles / 2;
  a.ptr = s->d_ptr;
  a.nbr = s->d_nbr;
  a.slot = reinterpret_cast<const typename SlotOf<R>::type *>(s->d_slot);
  a.inv_vol = reinterpret_cast<const R *>(s->d_inv_vol);
  a.wface = s->d_wface;
  a.gs = s->d_gs;
  a.gd = s->d_gd;
  a.kind = s->d_kind;
  a.aux = s->d_aux;
  a.bc_row = s->d_bc_row;
  a.I0 = reinterpret_cast<const R *>(s->d_I0);
  a.ext = s->d_ext;
  a.dir = reinterpret_cast<const R *>(s->d_dir);
  a.wt2 = reinterpret_cast<const R *>(s->d_wt);
  a.I_in = reinterpret_cast<const R *>(s->d_I[s->cur]);
  a.I_out = reinterpret_cast<R *>(s->d_I[s->cur ^ 1]);
  a.dt = dt;
  a.dt_r = R(dt);
  a.dt_cbar_r = R(dt * s->params.cbar);
  a.inv_c_r = R(1.0 / s->params.c);
  a.cellv = reinterpret_cast<R *>(s->d_cellv);
  a.cbar = s->params.cbar;
  a.c = s->params.c;
  a.a_rad = s->params.a_rad;
  a.rcv = s->params.r_gas / (s->params.gamma_gas - 1.0);
  a.k_dcr = dt * s->params.cbar;
  a.k_alpha = dt * s->params.c * s->params.a_rad;
  a.k_g = dt * s->params.c * 4.0 * kPi;
  a.k_fe = s->params.c / s->params.cbar * 4.0 * kPi;
  a.k_fm = 4.0 * kPi / s->params.cbar;
  a.newton_max_iter = s->params.newton_max_iter;
  a.status = s->d_status;
  a.bad_cell = s->d_bad;
  const unsigned blocks = (unsigned)((s->n_cells + CPB - 1) / CPB);
  step_kernel<R, PPT, MOVING, FULL><<<blocks, NT, 0, s->stream>>>(a);
  s->launches++;
  return cudaGetLastError();
}

template <typename R, bool MOVING, bool FULL> cudaError_t dispatch_ppt(rt_state *s, double dt) {
  const int ppt = (s->n_angles / 2 + KT - 1) / KT;
  switch (ppt) {
    case 1: return launch_t<R, 1, MOVING, FULL>(s, dt);
    case 2: return launch_t<R, 2, MOVING, FULL>(s, dt);
    case 3: return launch_t<R, 3, MOVING, FULL>(s, dt);
    case 4: return launch_t<R, 4, MOVING, FULL>(s, dt);
    case 5: return launch_t<R, 5, MOVING, FULL>(s, dt);
    case 6: return launch_t<R, 6, MOVING, FULL>(s, dt);
    case 7: return launch_t<R, 7, MOVING, FULL>(s, dt);
    case 8: return launch_t<R, 8, MOVING, FULL>(s, dt);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R> cudaError_t dispatch(rt_state *s, double dt) {
  const bool full = (s->n_angles / 2) % KT == 0;
  if (s->moving)
    return full ? dispatch_ppt<R, true, true>(s, dt) : dispatch_ppt<R, true, false>(s, dt);
  return full ? dispatch_ppt<R, false, true>(s, dt) : dispatch_ppt<R, false, false>(s, dt);
}

}  // namespace

cudaError_t launch_step(rt_state *s, double dt) {
  cudaError_t e = (s->precision == RT_FP32) ? dispatch<float>(s, dt) : dispatch<double>(s, dt);
  if (e == cudaSuccess) s->cur ^= 1;
  return e;
}

}  // namespace rt
