// Discrete adjoint of one radiation step (transport, Sec. 2.2, then the
// implicit comoving source, Sec. 2.3, with the boundary and emitter cells of
// Secs. 2.4-2.5), for gradients of a scalar loss with respect to the
// per-cell absorption opacities and the initial intensities.
//
//   I*  = M I^n                       (linear upwind transport)
//   (I^{n+1}, e^{n+1}, m^{n+1}) = S(I*, e^n, m^n; kappa_P, kappa_J)
//
// Reverse: the source adjoint per cell gives dL/dI*, dL/de^n, dL/dm^n and
// accumulates dL/dkappa; the transport adjoint applies M^T by a gather over
// the same face lists.  The temperature T^{n+1} is defined implicitly by
// alpha T^4 + rho c_v T - g = 0; its derivatives follow from the
// implicit-function theorem, dT/dalpha = -T^4 / F', dT/dg = 1 / F',
// F' = 4 alpha T^3 + rho c_v.
//
// Three launches (besides the permutes into and out of the internal order):
//   launch_transport (forward)  I* = M I^n, on the step kernel's tile machinery;
//   source_reverse_tile         blocks of 32 cells x 8 threads (the step
//                               kernel's tile mapping):
//     0  one lane per cell in double: the per-cell constants of phases 1 and
//        3 (v/c, x/Gamma, the boundary and emitter factors);
//     1  after a block barrier: the angular sums of the forward source step
//        and lambda_q = sum_a Gamma_a lambda_I~'_a / (1 + x_a), which needs
//        no result of the quartic;
//     2  after a second barrier, one lane per cell: the quartic, J~, q and
//        the reverse of the per-cell chain down to lambda_{S_I} and
//        lambda_{S_G} (in the state precision, see cell_chain);
//     3  after a third barrier, the per-angle reverse in the state precision,
//        written as L = dt/V lambda_I*.  The weight normalisation's sum
//        sum_a w~_a lambda_w~_a equals lambda_{S_I} S_I + lambda_{S_G} S_G, so
//        it needs no further pass over the angles;
//     4  after a fourth barrier, one lane per cell in double: lambda_e,
//        lambda_m and the opacity gradients from the cell sums of phase 3;
//   launch_transport (adjoint)  lambda_I^n = M^T lambda_I*: per cell,
//        lambda_c - sum over the faces with u > 0 of u (L_c - L_nbr).
// As in the forward step, the per-cell work is one lane per cell (GB300's
// FP64 rate is a small fraction of its FP32 rate) and the per-angle
// arithmetic runs in the state precision.
#include <cuda_runtime.h>

#include "rt_internal.cuh"
#include "rt_step_common.cuh"
#include "rt_step_tile.cuh"

namespace rt {
namespace {

using step::positive;
using step::rcp;

constexpr int kThreads = 256;  // threads per block of the per-cell gather / scatter

template <typename R> struct AdjArgs {
  int64_t n;
  int A, H, quad_end;
  const R *inv_vol;    // [N]
  const GasStatic *gs; // [N]
  const uint8_t *kind; // [N]
  const double2 *aux;  // [N] (tau or emit_rate, I_src)
  const R *dir;        // [A][4] (x, y, z, 0), caller angle order
  const R *wt2;        // [A/2][2] weights of the pairs (p, p + A/2)
  const R *Is;         // [N][A] I* (the transported rows)
  const R *lI1;        // [N][A] lambda_I^{n+1}
  R *Ls;               // [N][A] out: dt/V lambda_I*
  const double *e, *m, *le1, *lm1;  // [N], [N][3], [N], [N][3]
  double *le, *lm, *gP, *gJ;        // out: [N], [N][3]; gP, gJ accumulate
  double dt, cbar, c, a_rad, inv_c;
  R dt_r, k_ex_r;      // dt; 4 pi / cbar
  int newton_max_iter;
};

// 1 / v: float by the approximate reciprocal (v = Gamma or 1 + x Gamma,
// normal or +inf); double refined from it, or divided outside float range.
__device__ __forceinline__ float rcp_pos(float v) { return rcp(v); }
__device__ __forceinline__ double rcp_pos(double v) { return v < 1e37 ? rcp(v) : 1.0 / v; }

// Comoving quantities of one angle of an interior cell: Gamma = 1 - v.n/c,
// w^ = w / Gamma^2, r = 1 / (1 + x), x = X Gamma, I~ = Gamma^4 I*.
template <typename R> struct Ang {
  R G, iG, iG4, wh, r, It;
};
template <typename R> __device__ __forceinline__ Ang<R> comoving_g(R G, R wt, R X, R is) {
  Ang<R> g;
  g.G = G;
  g.iG = rcp_pos(g.G);
  const R iG2 = g.iG * g.iG, G2 = g.G * g.G;
  g.iG4 = iG2 * iG2;
  g.wh = wt * iG2;
  g.r = rcp_pos(fma(X, g.G, R(1)));
  g.It = G2 * G2 * is;
  return g;
}
// Per-cell inputs of phases 1 and 3 (phase 0), sums of phase 1 (unnormalised
// by N_w = sum w^), results of phase 2 and sums of phase 3.
template <typename R> struct CellIn {
  R bx, by, bz;  // v / c
  R X;           // interior: x / Gamma = dt cbar (rho kJ + rho kS); emitter: dt cbar (rho kappa)_src
  R f;           // boundary: 1 - min(dt / tau, 1); emitter: I_src
  R cle, lmx, lmy, lmz;  // c lambda_e, lambda_m of step n + 1
  int kind;
};
template <typename R> struct CellSums {
  R Nw, SI, SG, S1, lq;
};
template <typename R> struct CellRev {
  double gJ, lm[3];
  R q, lSI, lSG, swl, iNw;  // for phase 3
};
template <typename R> struct CellOut {
  R gJx, lvx, lvy, lvz;  // sum Gamma lambda_x; sum n lambda_Gamma (emitter: n dI'/dGamma lambda_I')
};

// Phase 0 for cell c.
template <typename R> __device__ void cell_inputs(const AdjArgs<R> &a, int64_t c, CellIn<R> &o) {
  const int kind = a.kind[c];
  const GasStatic &gs = a.gs[c];
  const double vc = gs.inv_rho * a.inv_c;
  o.kind = kind;
  o.bx = R(a.m[3 * c] * vc);
  o.by = R(a.m[3 * c + 1] * vc);
  o.bz = R(a.m[3 * c + 2] * vc);
  o.cle = R(a.c * a.le1[c]);
  o.lmx = R(a.lm1[3 * c]);
  o.lmy = R(a.lm1[3 * c + 1]);
  o.lmz = R(a.lm1[3 * c + 2]);
  o.X = R(a.dt * a.cbar * (gs.rkJ + gs.rkS));
  o.f = R(0);
  if (kind == RT_CELL_BOUNDARY) {
    const double2 ax = a.aux[c];
    o.f = R(1.0 - ((ax.x <= a.dt) ? 1.0 : a.dt / ax.x));
  } else if (kind == RT_CELL_EMITTER) {
    const double2 ax = a.aux[c];
    o.X = R(a.dt * a.cbar * ax.x);
    o.f = R(ax.y);
  }
}

// Phase 2 for one interior cell in the compute type C: the forward
// per-cell chain (the weights normalised, D = S_1 + dt cbar rho kJ S_G =
// 1 - dt cbar rho kS S_G) and its reverse from lambda_q down to lambda_{S_I},
// lambda_{S_G}.  The quartic is solved as in the forward step, from the gas
// temperature before the step.  Float states run it in float (the precision
// of their linearisation point; the forward float step solves its quartic in
// float too) and repeat it in double when a result is not finite; double
// states run it in double.
template <typename C> struct Chain {
  C q, lSI, lSG, swl, iNw, dle, lkin, gP, gJ;
};
template <typename C> __device__ __forceinline__ C tol_of();
template <> __device__ __forceinline__ float tol_of<float>() { return 1e-7f; }
template <> __device__ __forceinline__ double tol_of<double>() { return 1e-15; }

template <typename C, typename R>
__device__ Chain<C> cell_chain(const AdjArgs<R> &a, const GasStatic &gs, double eint,
                               const CellSums<R> &s) {
  Chain<C> o;
  const C iNw = C(1) / C(s.Nw);
  const C SI = C(s.SI) * iNw, SG = C(s.SG) * iNw, S1 = C(s.S1) * iNw, lq = C(s.lq);
  const C rho = C(gs.rho), ir = C(gs.inv_rho), rcv = C(gs.rcv), irc = C(1) / rcv;
  const C kP = C(gs.rkP) * ir, kJ = C(gs.rkJ) * ir, kS = C(gs.rkS) * ir;
  const C dcb = C(a.dt * a.cbar) * rho, dcc = C(a.dt * a.c) * rho, a_rad = C(a.a_rad);
  const C pi4 = C(4.0 * kPi);
  const C Tn = C(eint) * irc;
  const C D = S1 + dcb * kJ * SG;
  const C iD = C(1) / D;
  const C hJ = S1 * iD;  // 1 - dt cbar rho kJ S_G / D
  const C alpha = dcc * kP * a_rad * hJ;
  const C g = rcv * Tn + dcc * pi4 * kJ * SI * iD;
  C T;
  step::quartic_root(alpha, rcv, g, Tn, tol_of<C>(), a.newton_max_iter, &T);
  const C T3 = T * T * T, T4 = T3 * T;
  const C B = a_rad * T4 * C(0.25 / kPi);
  const C J = (SI + dcb * kP * B * SG) * iD;
  // reverse
  C gP = dcb * B * lq, gJ = C(0);
  C lB = dcb * kP * lq;
  const C lJ = dcb * kS * lq;
  C lSI = lJ * iD;
  C lSG = dcb * kP * B * lJ * iD;
  C lD = -J * lJ * iD;
  lB += dcb * kP * SG * lJ * iD;
  gP += dcb * B * SG * lJ * iD;
  const C lT = a_rad * T3 * C(1.0 / kPi) * lB;
  const C iFp = C(1) / (C(4) * alpha * T3 + rcv);
  const C lalpha = -T4 * iFp * lT;
  const C lg = lT * iFp;
  const C lTn = rcv * lg;
  lSI += dcc * pi4 * kJ * iD * lg;
  lD -= dcc * pi4 * kJ * SI * iD * iD * lg;
  gJ += dcc * pi4 * SI * iD * lg;
  gP += dcc * a_rad * hJ * lalpha;
  gJ -= dcc * kP * a_rad * dcb * SG * iD * lalpha;
  lSG -= dcc * kP * a_rad * dcb * kJ * iD * lalpha;
  lD += dcc * kP * a_rad * dcb * kJ * SG * iD * iD * lalpha;
  lSG -= dcb * kS * lD;
  o.q = dcb * (kP * B + kS * J);
  o.lSI = lSI;
  o.lSG = lSG;
  o.swl = lSI * SI + lSG * SG;
  o.iNw = iNw;
  o.dle = lTn * irc;  // lambda_e^n = lambda_e^{n+1} + lambda_Tn / rho c_v
  o.lkin = -o.dle;
  o.gP = gP;
  o.gJ = gJ;
  return o;
}

template <typename C> __device__ __forceinline__ bool chain_finite(const Chain<C> &o) {
  return isfinite(o.q) && isfinite(o.lSI) && isfinite(o.lSG) && isfinite(o.swl) &&
         isfinite(o.iNw) && isfinite(o.dle) && isfinite(o.gP) && isfinite(o.gJ);
}

// Phase 2 for cell c: the chain, lambda_e, the kappa_P gradient and the
// per-cell results phase 3 and phase 4 read.
template <typename R>
__device__ void cell_reverse(const AdjArgs<R> &a, int64_t c, const CellSums<R> &s,
                             CellRev<R> &r) {
  const GasStatic gs = a.gs[c];
  const double mx = a.m[3 * c], my = a.m[3 * c + 1], mz = a.m[3 * c + 2];
  const double eint = a.e[c] - 0.5 * (mx * mx + my * my + mz * mz) * gs.inv_rho;
  double q, lSI, lSG, swl, iNw, dle, lkin, gP, gJ;
  bool done = false;
  if constexpr (sizeof(R) == 4) {
    const Chain<float> o = cell_chain<float>(a, gs, eint, s);
    if (chain_finite(o)) {
      q = o.q, lSI = o.lSI, lSG = o.lSG, swl = o.swl, iNw = o.iNw;
      dle = o.dle, lkin = o.lkin, gP = o.gP, gJ = o.gJ;
      done = true;
    }
  }
  if (!done) {
    const Chain<double> o = cell_chain<double>(a, gs, eint, s);
    q = o.q, lSI = o.lSI, lSG = o.lSG, swl = o.swl, iNw = o.iNw;
    dle = o.dle, lkin = o.lkin, gP = o.gP, gJ = o.gJ;
  }
  a.le[c] = a.le1[c] + dle;
  a.gP[c] += gP;
  r.q = R(q);
  r.lSI = R(lSI);
  r.lSG = R(lSG);
  r.swl = R(swl);
  r.iNw = R(iNw);
  r.gJ = gJ;
  r.lm[0] = a.lm1[3 * c] + mx * gs.inv_rho * lkin;
  r.lm[1] = a.lm1[3 * c + 1] + my * gs.inv_rho * lkin;
  r.lm[2] = a.lm1[3 * c + 2] + mz * gs.inv_rho * lkin;
}

// Phase 4 for cell c: lambda_v = -(sum n lambda_Gamma) / c enters lambda_m
// through v = m / rho; the x_a = dt cbar rho (kJ + kS) Gamma_a term gives the
// kappa_J gradient.
template <typename R>
__device__ void cell_finish(const AdjArgs<R> &a, int64_t c, int kind, const CellRev<R> &r,
                            const CellOut<R> &s) {
  const double rho = a.gs[c].rho;
  const double f = -a.inv_c * a.gs[c].inv_rho;
  if (kind == RT_CELL_BOUNDARY) {
    a.le[c] = a.le1[c];
    for (int d = 0; d < 3; ++d) a.lm[3 * c + d] = a.lm1[3 * c + d];
  } else if (kind == RT_CELL_EMITTER) {
    a.le[c] = a.le1[c];
    a.lm[3 * c] = a.lm1[3 * c] + f * (double)s.lvx;
    a.lm[3 * c + 1] = a.lm1[3 * c + 1] + f * (double)s.lvy;
    a.lm[3 * c + 2] = a.lm1[3 * c + 2] + f * (double)s.lvz;
  } else {
    a.gJ[c] += r.gJ + a.dt * a.cbar * rho * (double)s.gJx;
    a.lm[3 * c] = r.lm[0] + f * (double)s.lvx;
    a.lm[3 * c + 1] = r.lm[1] + f * (double)s.lvy;
    a.lm[3 * c + 2] = r.lm[2] + f * (double)s.lvz;
  }
}

// ------------------------------------------------------------ the kernel
// Phases 1 and 3 (per angle) run on the step kernel's tile mapping: 32 cells
// x 8 threads, thread `sub` holding the entries of its pair / quad map (angle
// p and its antipode, whose Gamma is 1 + v.n_p where p's is 1 - v.n_p).  A
// cell's sums reduce over its 8 threads (3 shuffles), the 4 cells of a warp
// at once.  Phases 0, 2 and 4 run one lane per cell on warp 0.

// One angle's terms of phase 1 (interior cells).
template <typename R>
__device__ __forceinline__ void sums_angle(R G, R wt, R X, R is, R l1, R ex, R &Nw, R &SI, R &SG,
                                           R &S1, R &lq) {
  const Ang<R> g = comoving_g(G, wt, X, is);
  const R whr = g.wh * g.r;
  Nw += g.wh;
  SI = fma(whr, g.It, SI);
  SG = fma(whr, g.G, SG);
  S1 += whr;
  lq = fma(g.G * ((l1 - ex) * g.iG4), g.r, lq);
}

// One angle's terms of phase 3 (interior cells): returns dt/V lambda_I*,
// accumulates sum Gamma lambda_x and gives lambda_Gamma.
template <typename R>
__device__ __forceinline__ R reverse_angle(R G, R wt, R X, R isv, R l1, R ex, R dtv,
                                           const CellRev<R> &r, R &gJx, R &lGo) {
  const Ang<R> g = comoving_g(G, wt, X, isv);
  const R w = g.wh * r.iNw;
  const R Itn = fma(r.q, g.G, g.It) * g.r;  // I~'
  const R In = Itn * g.iG4;                 // I'
  const R lIn = l1 - ex;
  const R lItn = lIn * g.iG4;
  R lG = fma(R(-4) * In * g.iG, lIn, r.q * lItn * g.r);
  R lIt = lItn * g.r;
  R lx = -Itn * lItn * g.r;
  const R lw = fma(g.It, r.lSI, g.G * r.lSG) * g.r;  // lambda of the normalised weight
  lIt = fma(w * r.lSI, g.r, lIt);
  lG = fma(w * r.lSG, g.r, lG);
  lx = fma(-w * lw, g.r, lx);
  gJx = fma(g.G, lx, gJx);
  lG = fma(X, lx, lG);
  lG = fma(R(-2) * g.wh * g.iG, (lw - r.swl) * r.iNw, lG);
  const R G2 = g.G * g.G;
  lG = fma(R(4) * G2 * g.G * isv, lIt, lG);
  lGo = lG;
  return dtv * fma(G2 * G2, lIt, ex);
}

// One angle of an emitter cell: I' = (I* + Y I_src / Gamma^3) / (1 + Y Gamma);
// returns dt/V lambda_I* and gives dI'/dGamma lambda_I'.
template <typename R>
__device__ __forceinline__ R emitter_angle(R G, R Y, R isrc, R isv, R l1, R dtv, R &lGo) {
  const R iG = rcp_pos(G), iG2 = iG * iG, iG4 = iG2 * iG2, G2 = G * G;
  const R y = Y * G, iy = rcp_pos(R(1) + y);
  const R In = fma(G2 * G2, isv, y * isrc) * iy * iG4;
  const R dIdG = -fma(R(3) * Y * isrc, iG4, Y * In) * iy;  // dI'/dGamma
  lGo = dIdG * l1;
  return dtv * (l1 * iy);
}

// A thread's entries of one cell: directions and weights of its pairs, the
// rows of I* and lambda_I^{n+1} (padding entries: zero weights and rows).
template <typename R, typename M> struct Entries {
  R nx[M::PPT], ny[M::PPT], nz[M::PPT], wa[M::PPT], wb[M::PPT];
  R Ia[M::PPT], Ib[M::PPT], la[M::PPT], lb[M::PPT];
  __device__ __forceinline__ void load(const AdjArgs<R> &a, int64_t c, int sub, int np) {
#pragma unroll
    for (int j = 0; j < M::PPT; ++j) {
      const bool ok = M::FULL || j < np;
      const int p = ok ? M::pair(j, sub) : 0;
      step::load_dir(a.dir, p, nx[j], ny[j], nz[j]);
      wa[j] = ok ? a.wt2[2 * p] : R(0);
      wb[j] = ok ? a.wt2[2 * p + 1] : R(0);
    }
    M::load(a.Is + (size_t)c * a.A, sub, Ia, Ib, np);
    M::load(a.lI1 + (size_t)c * a.A, sub, la, lb, np);
  }
  // 4 pi w (c lambda_e + n . lambda_m) / cbar of entry j's angle (anti: the
  // antipode, direction -n_p)
  __device__ __forceinline__ R ex(int j, bool anti, const CellIn<R> &ci, R k_ex) const {
    const R x = anti ? -nx[j] : nx[j], y = anti ? -ny[j] : ny[j], z = anti ? -nz[j] : nz[j];
    return k_ex * (anti ? wb[j] : wa[j]) * fma(x, ci.lmx, fma(y, ci.lmy, fma(z, ci.lmz, ci.cle)));
  }
};

template <typename R> __device__ __forceinline__ R group_sum(R v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// Cells per block of the source reverse (8 threads each).
constexpr int kRevCells = CPB;
constexpr int kRevThreads = kRevCells * step::KT;

template <typename R, typename M>
__global__ void __launch_bounds__(kRevThreads, sizeof(R) == 4 ? (M::PPT <= 5 ? 4 : 3) : 2)
    source_reverse_tile(const AdjArgs<R> a) {
  using step::KT;
  constexpr int PPT = M::PPT;
  __shared__ CellIn<R> cin[kRevCells];
  __shared__ CellSums<R> sums[kRevCells];
  __shared__ CellRev<R> rev[kRevCells];
  __shared__ CellOut<R> cout_[kRevCells];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int lc = threadIdx.x / KT, sub = threadIdx.x % KT;
  const int64_t c0 = (int64_t)blockIdx.x * kRevCells;
  const int64_t cl = c0 + lane;  // the lane's cell in phases 0, 2, 4
  const bool lane_cell = warp == 0 && lane < kRevCells && cl < a.n;
  // ---------------- phase 0: per-cell constants, one lane per cell
  if (lane_cell) cell_inputs(a, cl, cin[lane]);

  const bool live = c0 + lc < a.n;
  const int64_t c = live ? c0 + lc : a.n - 1;  // dead threads shadow the last cell
  const int np = M::count(a.H, sub);
  __syncthreads();
  const CellIn<R> ci = cin[lc];
  const R k_ex = a.k_ex_r;  // lambda_I* gets 4 pi w (c lambda_e + n . lambda_m) / cbar
  // ---------------- phase 1: the angular sums and lambda_q
  {
    R Nw = 0, SI = 0, SG = 0, S1 = 0, lq = 0;
    if (ci.kind == RT_CELL_INTERIOR) {
      Entries<R, M> E;
      E.load(a, c, sub, np);
#pragma unroll
      for (int j = 0; j < PPT; ++j)
        if (M::FULL || j < np) {
          const R t = fma(ci.bx, E.nx[j], fma(ci.by, E.ny[j], ci.bz * E.nz[j]));
          sums_angle(R(1) - t, E.wa[j], ci.X, E.Ia[j], E.la[j], E.ex(j, false, ci, k_ex), Nw, SI,
                     SG, S1, lq);
          sums_angle(R(1) + t, E.wb[j], ci.X, E.Ib[j], E.lb[j], E.ex(j, true, ci, k_ex), Nw, SI,
                     SG, S1, lq);
        }
    }
    Nw = group_sum(Nw);
    SI = group_sum(SI);
    SG = group_sum(SG);
    S1 = group_sum(S1);
    lq = group_sum(lq);
    if (sub == 0) sums[lc] = CellSums<R>{Nw, SI, SG, S1, lq};
  }
  __syncthreads();

  // ---------------- phase 2: the quartic and the per-cell chain, one lane per cell
  if (lane_cell && cin[lane].kind == RT_CELL_INTERIOR) cell_reverse(a, cl, sums[lane], rev[lane]);
  __syncthreads();

  // ---------------- phase 3: per-angle reverse, lambda_I* (the entries read again: the
  // rows are in L1, and nothing per angle stays live across phase 2)
  {
    const R dtv = a.dt_r * a.inv_vol[c];  // the scale the adjoint transport divides out
    Entries<R, M> E;
    E.load(a, c, sub, np);
    R oa[PPT], ob[PPT];
    R gJx = 0, lvx = 0, lvy = 0, lvz = 0;
    if (ci.kind == RT_CELL_BOUNDARY) {
      const R f = dtv * ci.f;
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        oa[j] = f * E.la[j];
        ob[j] = f * E.lb[j];
      }
    } else if (ci.kind == RT_CELL_EMITTER) {
      const R Y = ci.X, isrc = ci.f;
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        const R t = fma(ci.bx, E.nx[j], fma(ci.by, E.ny[j], ci.bz * E.nz[j]));
        R ga = 0, gb = 0;
        oa[j] = emitter_angle(R(1) - t, Y, isrc, E.Ia[j], E.la[j], dtv, ga);
        ob[j] = emitter_angle(R(1) + t, Y, isrc, E.Ib[j], E.lb[j], dtv, gb);
        if (M::FULL || j < np) {
          const R d = ga - gb;  // n_p lambda_Gamma of p plus -n_p that of the antipode
          lvx = fma(E.nx[j], d, lvx);
          lvy = fma(E.ny[j], d, lvy);
          lvz = fma(E.nz[j], d, lvz);
        }
      }
    } else {
      const CellRev<R> r = rev[lc];
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        const R t = fma(ci.bx, E.nx[j], fma(ci.by, E.ny[j], ci.bz * E.nz[j]));
        R ga = 0, gb = 0, gxa = 0, gxb = 0;
        oa[j] = reverse_angle(R(1) - t, E.wa[j], ci.X, E.Ia[j], E.la[j], E.ex(j, false, ci, k_ex),
                              dtv, r, gxa, ga);
        ob[j] = reverse_angle(R(1) + t, E.wb[j], ci.X, E.Ib[j], E.lb[j], E.ex(j, true, ci, k_ex),
                              dtv, r, gxb, gb);
        if (M::FULL || j < np) {
          gJx += gxa + gxb;
          const R d = ga - gb;
          lvx = fma(E.nx[j], d, lvx);
          lvy = fma(E.ny[j], d, lvy);
          lvz = fma(E.nz[j], d, lvz);
        }
      }
    }
    if (live) M::store(a.Ls + (size_t)c * a.A, sub, oa, ob, np);
    gJx = group_sum(gJx);
    lvx = group_sum(lvx);
    lvy = group_sum(lvy);
    lvz = group_sum(lvz);
    if (sub == 0) cout_[lc] = CellOut<R>{gJx, lvx, lvy, lvz};
  }
  __syncthreads();

  // ---------------- phase 4: lambda_e, lambda_m, gradients, one lane per cell
  if (lane_cell) cell_finish(a, cl, cin[lane].kind, rev[lane], cout_[lane]);
}

template <typename R, typename M> void launch_reverse_tile(rt_state *s, const AdjArgs<R> &a) {
  const unsigned g = (unsigned)((s->n_cells + kRevCells - 1) / kRevCells);
  source_reverse_tile<R, M><<<g, kRevThreads, 0, s->stream>>>(a);
}

template <typename R, bool FULL> void reverse_pairs(rt_state *s, const AdjArgs<R> &a) {
  using step::PairMap;
  switch ((s->n_angles / 2 + step::KT - 1) / step::KT) {
    case 1: return launch_reverse_tile<R, PairMap<R, 1, FULL>>(s, a);
    case 2: return launch_reverse_tile<R, PairMap<R, 2, FULL>>(s, a);
    case 3: return launch_reverse_tile<R, PairMap<R, 3, FULL>>(s, a);
    case 4: return launch_reverse_tile<R, PairMap<R, 4, FULL>>(s, a);
    case 5: return launch_reverse_tile<R, PairMap<R, 5, FULL>>(s, a);
    case 6: return launch_reverse_tile<R, PairMap<R, 6, FULL>>(s, a);
    case 7: return launch_reverse_tile<R, PairMap<R, 7, FULL>>(s, a);
    default: return launch_reverse_tile<R, PairMap<R, 8, FULL>>(s, a);
  }
}

template <typename R> void launch_reverse(rt_state *s, const AdjArgs<R> &a) {
  using step::QuadMap;
  if constexpr (sizeof(R) == 4) {
    if (s->quad_end > 0) {  // rows in the quad layout
      switch (s->n_angles / 16) {
        case 2: return launch_reverse_tile<float, QuadMap<1, false>>(s, a);
        case 3: return launch_reverse_tile<float, QuadMap<1, true>>(s, a);
        case 4: return launch_reverse_tile<float, QuadMap<2, false>>(s, a);
        case 5: return launch_reverse_tile<float, QuadMap<2, true>>(s, a);
        case 6: return launch_reverse_tile<float, QuadMap<3, false>>(s, a);
        case 7: return launch_reverse_tile<float, QuadMap<3, true>>(s, a);
        default: return launch_reverse_tile<float, QuadMap<4, false>>(s, a);
      }
    }
  }
  if ((s->n_angles / 2) % step::KT == 0)
    reverse_pairs<R, true>(s, a);
  else
    reverse_pairs<R, false>(s, a);
}

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
  R *Ls = reinterpret_cast<R *>(s->d_adj[1]);
  cudaError_t err = launch_transport(s, dt, I_int, Is, false);
  if (err != cudaSuccess) return err;
  AdjArgs<R> a;
  a.n = N;
  a.A = A;
  a.H = A / 2;
  a.quad_end = s->quad_end;
  a.inv_vol = reinterpret_cast<const R *>(s->d_inv_vol);
  a.gs = s->d_gs;
  a.kind = s->d_kind;
  a.aux = s->d_aux;
  a.dir = reinterpret_cast<const R *>(s->d_dir);
  a.wt2 = reinterpret_cast<const R *>(s->d_wt);
  a.Is = Is;
  a.lI1 = lI1_int;
  a.Ls = Ls;
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
  a.inv_c = 1.0 / s->params.c;
  a.dt_r = R(dt);
  a.k_ex_r = R(4.0 * kPi / s->params.cbar);
  a.newton_max_iter = s->params.newton_max_iter;
  launch_reverse<R>(s, a);
  s->launches++;
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_transport(s, dt, Ls, lI_int, true);
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
