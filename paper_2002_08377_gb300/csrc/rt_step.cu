// Fused radiation step: upwind transport (Sec. 3.2) + implicit comoving
// source update with gas exchange (Sec. 3.3), boundary cells (Sec. 3.5) and
// emitter cells (Sec. 3.6), one kernel per step.
//
// Block = 32 cells x 8 threads.  Thread `sub` of a cell owns the angle pairs
// p = sub + 8 j (j < PPT) and their antipodes p + A/2; the flux coefficient
// of the antipode through a face is u(p + A/2) = -(n_p . s) - w, so one dot
// product serves two angles and, on a static mesh, exactly one of the two
// needs the neighbour's value.  The face sum runs in the cell's slot order
// (no atomics, deterministic).
//
// Phases (separated by __syncthreads):
//   A  all threads: transport, comoving weights, angular sums (precision R);
//      each cell's 8 lanes reduce with shuffles into shared memory;
//   B  warp 0, one lane per cell: the gas temperature quartic in double
//      (FP32 states start Newton from a float estimate);
//   C  all threads: new intensities, store, radiation change per cell;
//   D  warp 0, one lane per cell: gas energy / momentum (or tally) update in
//      double.
// Keeping the double-precision work lane-per-cell matters on GB300, whose
// FP64 rate is a small fraction of its FP32 rate.
#include <cuda_runtime.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int KT = 8;            // threads per cell
constexpr int CPB = 32;          // cells per block
constexpr int NT = KT * CPB;     // threads per block

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

// Reciprocal: the correctly rounded float reciprocal, or in double the
// float estimate refined by two Newton steps (|error| ~ 1 ulp); arguments
// here are 1 + x (x >= 0) and Gamma^2, well inside float range.
template <typename R> __device__ __forceinline__ R rcp(R x);
template <> __device__ __forceinline__ float rcp<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double rcp<double>(double x) {
  double r = (double)__frcp_rn((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
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

// Positive root of alpha T^4 + beta T = g (alpha >= 0, beta > 0, g >= 0).
// f is increasing and convex on T > 0, so Newton from any point at or above
// the root decreases monotonically onto it; it stops when an iterate fails
// to decrease or moves by at most 1e-15 of itself.  FLOAT_START: a float
// Newton estimate plus one unconditional double step (which lands at or
// above the root by convexity) replaces the start min(g/beta, (g/alpha)^.25).
// Positive root of alpha T^4 + beta T = g (alpha >= 0, beta > 0, g >= 0).
// f is increasing and convex on T > 0, so Newton from any point at or above
// the root decreases monotonically onto it.  Double states: start at
// min(g/beta, (g/alpha)^(1/4)) and stop when an iterate fails to decrease or
// moves by at most 1e-15 of itself.  Float states: the same iteration in
// float to a relative 1e-7, then one Newton step in double (the float
// root's error ~1e-7 becomes ~1e-14).  Returns 1 if the iteration did not
// converge within max_iter.
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
      double r = (double)__frcp_rn((float)fp);
      r = fma(r, fma(-fp, r, 1.0), r);
      *T_out = fma(-f, r, T);
      return 0;
    }
    // coefficients outside float range: solve in double below
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

constexpr int MAXS = 1024;  // face slots a block stages in shared memory

template <typename R> struct Shared {
  typename SlotOf<R>::type slot[MAXS];  // the block's face slots, in slot order
  int32_t nbr[MAXS];
  R ws[CPB], sI[CPB], sG[CPB];  // comoving weight sum and the two sums of Eq. (Jcom)
  R q[CPB];                     // dt cbar rho (kP B + kS J) per interior cell
  R dE[CPB], dF[3][CPB];        // sum w (I* - I') and sum w n (I* - I')
  unsigned bad[CPB];
};

// sum_f u I_up over slots [k0, k1) of one cell, for the thread's angle pairs
template <typename R, int PPT, bool MOVING, typename S>
__device__ __forceinline__ void face_sum(const S *__restrict__ slot, const int32_t *__restrict__ nbr,
                                         int64_t k0, int64_t k1, const R *__restrict__ I_in, int A,
                                         int H, int sub, const R (&nx)[PPT], const R (&ny)[PPT],
                                         const R (&nz)[PPT], const R (&Ia)[PPT],
                                         const R (&Ib)[PPT], R (&acca)[PPT], R (&accb)[PPT]) {
#pragma unroll 2
  for (int64_t k = k0; k < k1; ++k) {
    const int32_t nb = nbr[k];
    const S s = slot[k];
    const R *In = I_in + (size_t)nb * A;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int p = sub + KT * j;
      if (p < H) {
        const R d = fma(nx[j], s.sx, fma(ny[j], s.sy, nz[j] * s.sz));
        if (MOVING) {
          const R ua = d - s.w, ub = -d - s.w;
          R va = Ia[j], vb = Ib[j];
          if (ua < R(0)) va = __ldg(In + p);
          if (ub < R(0)) vb = __ldg(In + p + H);
          acca[j] = fma(ua, va, acca[j]);
          accb[j] = fma(ub, vb, accb[j]);
        } else {
          // u_a = d, u_b = -d: the inflow side of the pair reads the neighbour
          const bool out = d > R(0);
          const R v = __ldg(In + (out ? p + H : p));
          acca[j] = fma(d, out ? Ia[j] : v, acca[j]);
          accb[j] = fma(-d, out ? v : Ib[j], accb[j]);
        }
      }
    }
  }
}

template <typename R, int PPT, bool MOVING>
__global__ void __launch_bounds__(NT) step_kernel(const StepArgs<R> a) {
  __shared__ Shared<R> sh;
  const int lc = threadIdx.x / KT;
  const int sub = threadIdx.x % KT;
  const int64_t cell = (int64_t)blockIdx.x * CPB + lc;
  const bool live = cell < a.n_cells;
  const int64_t c = live ? cell : a.n_cells - 1;  // dead lanes shadow the last cell
  const int A = a.n_angles, H = a.half;

  // ---------------- phase A: transport, I* = I - dt/V sum_f u I_up
  R nx[PPT], ny[PPT], nz[PPT], Ia[PPT], Ib[PPT], acca[PPT], accb[PPT];
  const R *Ic = a.I_in + (size_t)c * A;
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int p = sub + KT * j;
    const bool v = p < H;
    const int pp = v ? p : 0;
    nx[j] = a.dir[4 * pp];
    ny[j] = a.dir[4 * pp + 1];
    nz[j] = a.dir[4 * pp + 2];
    Ia[j] = v ? Ic[pp] : R(0);
    Ib[j] = v ? Ic[pp + H] : R(0);
    acca[j] = R(0);
    accb[j] = R(0);
  }
  // stage the block's face slots (contiguous: cells are consecutive)
  const int64_t cb0 = (int64_t)blockIdx.x * CPB;
  const int64_t cb1 = cb0 + CPB < a.n_cells ? cb0 + CPB : a.n_cells;
  const int64_t kb = a.ptr[cb0];
  const int64_t cnt = a.ptr[cb1] - kb;
  const bool staged = cnt <= MAXS;  // uniform over the block
  if (staged) {
    for (int i = threadIdx.x; i < cnt; i += NT) {
      sh.slot[i] = load_slot<R>(a.slot + kb + i);
      sh.nbr[i] = __ldg(a.nbr + kb + i);
    }
  }
  __syncthreads();
  if (staged)
    face_sum<R, PPT, MOVING>(sh.slot, sh.nbr, a.ptr[c] - kb, a.ptr[c + 1] - kb, a.I_in, A, H, sub,
                             nx, ny, nz, Ia, Ib, acca, accb);
  else
    face_sum<R, PPT, MOVING>(a.slot, a.nbr, a.ptr[c], a.ptr[c + 1], a.I_in, A, H, sub, nx, ny, nz,
                             Ia, Ib, acca, accb);
  const R dtv = a.dt_r * a.inv_vol[c];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    Ia[j] = fma(-dtv, acca[j], Ia[j]);  // I* (zero for unused slots)
    Ib[j] = fma(-dtv, accb[j], Ib[j]);
  }

  // comoving frame (first order in v/c): Gamma = 1 -+ v.n / c, with the
  // cell's velocity and rho (kJ + kS) kept in the state precision
  const int kind = a.kind[c];
  const R vx = a.cellv[4 * c], vy = a.cellv[4 * c + 1], vz = a.cellv[4 * c + 2];
  const R xs = a.dt_cbar_r * a.cellv[4 * c + 3];
  const R inv_c = a.inv_c_r;
  R Ga[PPT], Gb[PPT];
  R ws = 0, sI = 0, sG = 0;
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int p = sub + KT * j;
    const R vn = (vx * nx[j] + vy * ny[j] + vz * nz[j]) * inv_c;
    Ga[j] = R(1) - vn;
    Gb[j] = R(1) + vn;
    if (p < H) {
      const R Ga2 = Ga[j] * Ga[j], Gb2 = Gb[j] * Gb[j];
      const R wca = a.wt[p] * rcp(Ga2), wcb = a.wt[p + H] * rcp(Gb2);
      const R ra = rcp(R(1) + xs * Ga[j]), rb = rcp(R(1) + xs * Gb[j]);
      ws += wca + wcb;
      sI += wca * (Ga2 * Ga2 * Ia[j]) * ra + wcb * (Gb2 * Gb2 * Ib[j]) * rb;
      sG += wca * Ga[j] * ra + wcb * Gb[j] * rb;
    }
  }
  ws = cell_sum(ws);
  sI = cell_sum(sI);
  sG = cell_sum(sG);
  if (sub == 0) {
    sh.ws[lc] = ws;
    sh.sI[lc] = sI;
    sh.sG[lc] = sG;
  }
  __syncthreads();

  // ---------------- phase B: temperature quartic, one lane per cell
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (warp == 0) {
    const int64_t cl = (int64_t)blockIdx.x * CPB + lane;
    R q = 0;
    unsigned bad = 0;
    if (cl < a.n_cells && a.kind[cl] == RT_CELL_INTERIOR) {
      const GasStatic g = a.gs[cl];
      const GasDyn d = a.gd[cl];
      const R iw = R(1) / sh.ws[lane];
      const double SI = (double)(sh.sI[lane] * iw), SG = (double)(sh.sG[lane] * iw);
      const double dcr = a.dt * a.cbar * g.rho;
      const double D = 1.0 - dcr * g.kS * SG;
      const double rD = 1.0 / D;
      const double kin = 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * g.inv_rho;
      const double Tn = (d.e - kin) * g.inv_rcv;
      const double alpha = a.dt * a.c * g.rho * g.kP * a.a_rad * (1.0 - dcr * g.kJ * SG * rD);
      const double gq = g.rcv * Tn + a.dt * a.c * g.rho * 4.0 * kPi * g.kJ * SI * rD;
      double T = 0.0;
      if (!(gq >= 0.0) || !(alpha >= 0.0)) {
        bad |= ST_NONFINITE;
      } else if (quartic_root<sizeof(R) == 4>(alpha, g.rcv, gq, a.newton_max_iter, &T)) {
        bad |= ST_NONCONV;
      }
      const double B = a.a_rad * (T * T) * (T * T) * (1.0 / (4.0 * kPi));
      const double J = (SI + dcr * g.kP * B * SG) * rD;
      q = R(dcr * (g.kP * B + g.kS * J));
    }
    sh.q[lane] = q;
    sh.bad[lane] = bad;
  }
  __syncthreads();

  // ---------------- phase C: new intensities and the radiation change
  R In_a[PPT], In_b[PPT];
  if (kind == RT_CELL_BOUNDARY) {
    const double2 ax = a.aux[c];
    const R f = R((ax.x <= a.dt) ? 1.0 : a.dt / ax.x);
    const R *I0 = a.I0 + (size_t)a.bc_row[c] * A;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int p = sub + KT * j;
      const bool v = p < H;
      In_a[j] = v ? fma(-f, Ia[j] - I0[p], Ia[j]) : R(0);
      In_b[j] = v ? fma(-f, Ib[j] - I0[p + H], Ib[j]) : R(0);
    }
  } else if (kind == RT_CELL_EMITTER) {
    const double2 ax = a.aux[c];
    const R ys = R(a.dt * a.cbar * ax.x);
    const R isrc = R(ax.y);
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const R Ga2 = Ga[j] * Ga[j], Gb2 = Gb[j] * Gb[j];
      const R Ga4 = Ga2 * Ga2, Gb4 = Gb2 * Gb2;
      const R ya = ys * Ga[j], yb = ys * Gb[j];
      In_a[j] = (Ga4 * Ia[j] + ya * isrc) * rcp((R(1) + ya) * Ga4);
      In_b[j] = (Gb4 * Ib[j] + yb * isrc) * rcp((R(1) + yb) * Gb4);
    }
  } else {
    const R q = sh.q[lc];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const R Ga2 = Ga[j] * Ga[j], Gb2 = Gb[j] * Gb[j];
      const R Ga4 = Ga2 * Ga2, Gb4 = Gb2 * Gb2;
      In_a[j] = (Ga4 * Ia[j] + q * Ga[j]) * rcp((R(1) + xs * Ga[j]) * Ga4);
      In_b[j] = (Gb4 * Ib[j] + q * Gb[j]) * rcp((R(1) + xs * Gb[j]) * Gb4);
    }
  }
  R de = 0, dfx = 0, dfy = 0, dfz = 0;
  unsigned nonfinite = 0;
  R *Io = a.I_out + (size_t)c * A;
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int p = sub + KT * j;
    if (p < H) {
      if (live) {
        Io[p] = In_a[j];
        Io[p + H] = In_b[j];
      }
      if (!isfinite(In_a[j]) || !isfinite(In_b[j])) nonfinite = ST_NONFINITE;
      const R da = a.wt[p] * (Ia[j] - In_a[j]);
      const R db = a.wt[p + H] * (Ib[j] - In_b[j]);
      de += da + db;
      const R dd = da - db;  // the antipode has direction -n
      dfx = fma(nx[j], dd, dfx);
      dfy = fma(ny[j], dd, dfy);
      dfz = fma(nz[j], dd, dfz);
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
  if (warp == 0) {
    const int64_t cl = (int64_t)blockIdx.x * CPB + lane;
    if (cl < a.n_cells) {
      const double fe = a.c / a.cbar * 4.0 * kPi;
      const double fm = 4.0 * kPi / a.cbar;  // (4 pi c sum w n dI) / (c cbar)
      const double dE = fe * (double)sh.dE[lane];
      const double dx = fm * (double)sh.dF[0][lane], dy = fm * (double)sh.dF[1][lane],
                   dz = fm * (double)sh.dF[2][lane];
      if (a.kind[cl] == RT_CELL_INTERIOR) {
        GasDyn d = a.gd[cl];
        d.e += dE;
        d.mx += dx;
        d.my += dy;
        d.mz += dz;
        a.gd[cl] = d;
        const double ir = a.gs[cl].inv_rho;  // frame velocity of the next step
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
}

template <typename R, int PPT, bool MOVING> cudaError_t launch_t(rt_state *s, double dt) {
  StepArgs<R> a;
  a.n_cells = s->n_cells;
  a.n_angles = s->n_angles;
  a.half = s->n_angles / 2;
  a.ptr = s->d_ptr;
  a.nbr = s->d_nbr;
  a.slot = reinterpret_cast<const typename SlotOf<R>::type *>(s->d_slot);
  a.inv_vol = reinterpret_cast<const R *>(s->d_inv_vol);
  a.gs = s->d_gs;
  a.gd = s->d_gd;
  a.kind = s->d_kind;
  a.aux = s->d_aux;
  a.bc_row = s->d_bc_row;
  a.I0 = reinterpret_cast<const R *>(s->d_I0);
  a.ext = s->d_ext;
  a.dir = reinterpret_cast<const R *>(s->d_dir);
  a.wt = reinterpret_cast<const R *>(s->d_wt);
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
  a.newton_max_iter = s->params.newton_max_iter;
  a.status = s->d_status;
  a.bad_cell = s->d_bad;
  const unsigned blocks = (unsigned)((s->n_cells + CPB - 1) / CPB);
  step_kernel<R, PPT, MOVING><<<blocks, NT, 0, s->stream>>>(a);
  s->launches++;
  return cudaGetLastError();
}

template <typename R, bool MOVING> cudaError_t dispatch_ppt(rt_state *s, double dt) {
  const int ppt = (s->n_angles / 2 + KT - 1) / KT;
  switch (ppt) {
    case 1: return launch_t<R, 1, MOVING>(s, dt);
    case 2: return launch_t<R, 2, MOVING>(s, dt);
    case 3: return launch_t<R, 3, MOVING>(s, dt);
    case 4: return launch_t<R, 4, MOVING>(s, dt);
    case 5: return launch_t<R, 5, MOVING>(s, dt);
    case 6: return launch_t<R, 6, MOVING>(s, dt);
    case 7: return launch_t<R, 7, MOVING>(s, dt);
    case 8: return launch_t<R, 8, MOVING>(s, dt);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R> cudaError_t dispatch(rt_state *s, double dt) {
  return s->moving ? dispatch_ppt<R, true>(s, dt) : dispatch_ppt<R, false>(s, dt);
}

}  // namespace

cudaError_t launch_step(rt_state *s, double dt) {
  cudaError_t e = (s->precision == RT_FP32) ? dispatch<float>(s, dt) : dispatch<double>(s, dt);
  if (e == cudaSuccess) s->cur ^= 1;
  return e;
}

}  // namespace rt
