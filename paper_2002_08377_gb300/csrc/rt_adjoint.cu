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
//   source_reverse_kernel       blocks of 32 cells, 4 per warp, lanes over the
//                               row positions of a cell:
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

namespace rt {
namespace {

using step::positive;
using step::rcp;

constexpr int kWarps = 8;                        // warps per block
constexpr int kCellsPerWarp = 4;                 // cells a warp takes in turn
constexpr int kCells = kWarps * kCellsPerWarp;   // cells per block
constexpr int kThreads = 32 * kWarps;

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

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

// The angles of one lane's row positions q = lane + 32 t.
template <typename R, int NT> struct Lane {
  R nx[NT], ny[NT], nz[NT], wt[NT];
  int q[NT];  // row position (>= A: none)
};

template <typename R, int NT>
__device__ __forceinline__ Lane<R, NT> lane_angles(const AdjArgs<R> &a, int lane) {
  Lane<R, NT> L;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int q = lane + 32 * t;
    L.q[t] = q;
    L.nx[t] = L.ny[t] = L.nz[t] = L.wt[t] = R(0);
    if (q < a.A) {
      const int an = angle_of_position(q, a.H, a.quad_end);
      const int p = an < a.H ? an : an - a.H;
      L.nx[t] = a.dir[4 * an];
      L.ny[t] = a.dir[4 * an + 1];
      L.nz[t] = a.dir[4 * an + 2];
      L.wt[t] = a.wt2[2 * p + (an >= a.H ? 1 : 0)];
    }
  }
  return L;
}

// 1 / v: float by the approximate reciprocal (v = Gamma or 1 + x Gamma,
// normal or +inf); double refined from it, or divided outside float range.
__device__ __forceinline__ float rcp_pos(float v) { return rcp(v); }
__device__ __forceinline__ double rcp_pos(double v) { return v < 1e37 ? rcp(v) : 1.0 / v; }

// Comoving quantities of one angle of an interior cell: Gamma = 1 - v.n/c,
// w^ = w / Gamma^2, r = 1 / (1 + x), x = X Gamma, I~ = Gamma^4 I*.
template <typename R> struct Ang {
  R G, iG, iG4, wh, r, It;
};
template <typename R>
__device__ __forceinline__ Ang<R> comoving(R bx, R by, R bz, R nx, R ny, R nz, R wt, R X, R is) {
  Ang<R> g;
  g.G = R(1) - fma(bx, nx, fma(by, ny, bz * nz));
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

template <typename R, int NT>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 3 : 2)
    source_reverse_kernel(const AdjArgs<R> a) {
  __shared__ CellIn<R> cin[kCells];
  __shared__ CellSums<R> sums[kCells];
  __shared__ CellRev<R> rev[kCells];
  __shared__ CellOut<R> cout_[kCells];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t c0 = (int64_t)blockIdx.x * kCells;
  const int64_t cl = c0 + lane;  // the lane's cell in phases 0, 2, 4
  const bool lane_cell = warp == 0 && cl < a.n;

  // ---------------- phase 0: per-cell constants, one lane per cell
  if (lane_cell) cell_inputs(a, cl, cin[lane]);
  __syncthreads();

  const Lane<R, NT> L = lane_angles<R, NT>(a, lane);
  const R k_ex = a.k_ex_r;  // lambda_I* gets 4 pi w (c lambda_e + n . lambda_m) / cbar
  R is[kCellsPerWarp][NT];

  // ---------------- phase 1: the angular sums and lambda_q
#pragma unroll
  for (int i = 0; i < kCellsPerWarp; ++i) {
    const int64_t c = c0 + warp * kCellsPerWarp + i;
#pragma unroll
    for (int t = 0; t < NT; ++t)
      is[i][t] = c < a.n && L.q[t] < a.A ? a.Is[(size_t)c * a.A + L.q[t]] : R(0);
  }
#pragma unroll
  for (int i = 0; i < kCellsPerWarp; ++i) {
    const int lc = warp * kCellsPerWarp + i;
    const int64_t c = c0 + lc;
    if (c >= a.n) continue;
    const CellIn<R> &ci = cin[lc];
    if (ci.kind != RT_CELL_INTERIOR) continue;
    R Nw = 0, SI = 0, SG = 0, S1 = 0, lq = 0;
#pragma unroll
    for (int t = 0; t < NT; ++t)
      if (L.q[t] < a.A) {
        const Ang<R> g =
            comoving(ci.bx, ci.by, ci.bz, L.nx[t], L.ny[t], L.nz[t], L.wt[t], ci.X, is[i][t]);
        const R whr = g.wh * g.r;
        Nw += g.wh;
        SI = fma(whr, g.It, SI);
        SG = fma(whr, g.G, SG);
        S1 += whr;
        const R ex = k_ex * L.wt[t] *
                     fma(L.nx[t], ci.lmx, fma(L.ny[t], ci.lmy, fma(L.nz[t], ci.lmz, ci.cle)));
        const R l1 = a.lI1[(size_t)c * a.A + L.q[t]];
        lq = fma(g.G * ((l1 - ex) * g.iG4), g.r, lq);
      }
    Nw = warp_sum(Nw);
    SI = warp_sum(SI);
    SG = warp_sum(SG);
    S1 = warp_sum(S1);
    lq = warp_sum(lq);
    if (lane == 0) sums[lc] = CellSums<R>{Nw, SI, SG, S1, lq};
  }
  __syncthreads();

  // ---------------- phase 2: the quartic and the per-cell chain, one lane per cell
  if (lane_cell && cin[lane].kind == RT_CELL_INTERIOR) cell_reverse(a, cl, sums[lane], rev[lane]);
  __syncthreads();

  // ---------------- phase 3: per-angle reverse, lambda_I*
#pragma unroll
  for (int i = 0; i < kCellsPerWarp; ++i) {
    const int lc = warp * kCellsPerWarp + i;
    const int64_t c = c0 + lc;
    if (c >= a.n) continue;
    const CellIn<R> &ci = cin[lc];
    const R *l1row = a.lI1 + (size_t)c * a.A;
    R *out = a.Ls + (size_t)c * a.A;
    const R dtv = a.dt_r * a.inv_vol[c];  // the scale the adjoint transport divides out
    if (ci.kind == RT_CELL_BOUNDARY) {
      const R f = dtv * ci.f;
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (L.q[t] < a.A) out[L.q[t]] = f * l1row[L.q[t]];
      continue;
    }
    R gJx = 0, lvx = 0, lvy = 0, lvz = 0;
    if (ci.kind == RT_CELL_EMITTER) {
      // I' = (I* + Y I_src / Gamma^3) / (1 + Y Gamma), Y = dt cbar (rho kappa)_src
      const R Y = ci.X, isrc = ci.f;
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (L.q[t] < a.A) {
          const R G = R(1) - fma(ci.bx, L.nx[t], fma(ci.by, L.ny[t], ci.bz * L.nz[t]));
          const R iG = rcp_pos(G), iG2 = iG * iG, iG4 = iG2 * iG2, G2 = G * G;
          const R y = Y * G, iy = rcp_pos(R(1) + y);
          const R In = fma(G2 * G2, is[i][t], y * isrc) * iy * iG4;
          const R l1 = l1row[L.q[t]];
          out[L.q[t]] = dtv * (l1 * iy);
          const R dIdG = -fma(R(3) * Y * isrc, iG4, Y * In) * iy;  // dI'/dGamma
          lvx = fma(L.nx[t] * dIdG, l1, lvx);
          lvy = fma(L.ny[t] * dIdG, l1, lvy);
          lvz = fma(L.nz[t] * dIdG, l1, lvz);
        }
    } else {
      const CellRev<R> &r = rev[lc];
      const R q = r.q, lSI = r.lSI, lSG = r.lSG, swl = r.swl, iNw = r.iNw;
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (L.q[t] < a.A) {
          const R isv = is[i][t];
          const Ang<R> g =
              comoving(ci.bx, ci.by, ci.bz, L.nx[t], L.ny[t], L.nz[t], L.wt[t], ci.X, isv);
          const R w = g.wh * iNw;
          const R Itn = fma(q, g.G, g.It) * g.r;  // I~'
          const R In = Itn * g.iG4;                // I'
          const R ex = k_ex * L.wt[t] *
                       fma(L.nx[t], ci.lmx, fma(L.ny[t], ci.lmy, fma(L.nz[t], ci.lmz, ci.cle)));
          const R lIn = l1row[L.q[t]] - ex;
          const R lItn = lIn * g.iG4;
          R lG = fma(R(-4) * In * g.iG, lIn, q * lItn * g.r);
          R lIt = lItn * g.r;
          R lx = -Itn * lItn * g.r;
          const R lw = fma(g.It, lSI, g.G * lSG) * g.r;  // lambda of the normalised weight
          lIt = fma(w * lSI, g.r, lIt);
          lG = fma(w * lSG, g.r, lG);
          lx = fma(-w * lw, g.r, lx);
          gJx = fma(g.G, lx, gJx);
          lG = fma(ci.X, lx, lG);
          lG = fma(R(-2) * g.wh * g.iG, (lw - swl) * iNw, lG);
          const R G2 = g.G * g.G;
          out[L.q[t]] = dtv * fma(G2 * G2, lIt, ex);
          lG = fma(R(4) * G2 * g.G * isv, lIt, lG);
          lvx = fma(L.nx[t], lG, lvx);
          lvy = fma(L.ny[t], lG, lvy);
          lvz = fma(L.nz[t], lG, lvz);
        }
    }
    gJx = warp_sum(gJx);
    lvx = warp_sum(lvx);
    lvy = warp_sum(lvy);
    lvz = warp_sum(lvz);
    if (lane == 0) cout_[lc] = CellOut<R>{gJx, lvx, lvy, lvz};
  }
  __syncthreads();

  // ---------------- phase 4: lambda_e, lambda_m, gradients, one lane per cell
  if (lane_cell) cell_finish(a, cl, cin[lane].kind, rev[lane], cout_[lane]);
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
  const unsigned g = (unsigned)((N + kCells - 1) / kCells);
  switch ((A + 31) / 32) {
    case 1: source_reverse_kernel<R, 1><<<g, kThreads, 0, s->stream>>>(a); break;
    case 2: source_reverse_kernel<R, 2><<<g, kThreads, 0, s->stream>>>(a); break;
    case 3: source_reverse_kernel<R, 3><<<g, kThreads, 0, s->stream>>>(a); break;
    default: source_reverse_kernel<R, 4><<<g, kThreads, 0, s->stream>>>(a); break;
  }
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
