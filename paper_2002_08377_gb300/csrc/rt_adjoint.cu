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
// Launches (besides the permutes of the rows into and out of the internal
// order):
//   adjoint_prep  one thread per cell, in double: gathers e^n, m^n,
//        lambda_e^{n+1}, lambda_m^{n+1} from the caller's order and writes
//        the cell's record: v/c, x/Gamma, the boundary and emitter factors,
//        c lambda_e, lambda_m and the inputs of the per-cell chain (rho,
//        1/rho, rho c_v, the opacities, the gas temperature before the step)
//        in the state precision;
//   launch_transport (forward)  I* = M I^n, on the step kernel's tile machinery;
//   source_reverse_tile  blocks of 32 cells x 8 threads (the step kernel's
//        tile mapping):
//     1  the angular sums of the forward source step and
//        lambda_q = sum_a Gamma_a lambda_I~'_a / (1 + x_a), which needs no
//        result of the quartic, reduced over the cell's 8 threads;
//     2  the quartic, J~, q and the reverse of the per-cell chain down to
//        lambda_{S_I} and lambda_{S_G}: float states in every thread of the
//        cell (the sums are in all 8, no block barrier); double states one
//        lane per cell on warp 0 between two block barriers, so that the FP64
//        chain is issued once for 32 cells;
//     3  the per-angle reverse in the state precision, written as
//        L = dt/V lambda_I*.  The weight normalisation's sum
//        sum_a w~_a lambda_w~_a equals lambda_{S_I} S_I + lambda_{S_G} S_G, so
//        it needs no further pass over the angles; the cell's sums of this
//        phase and the chain's results go to a per-cell record;
//   launch_transport (adjoint)  lambda_I^n = M^T lambda_I*: per cell,
//        lambda_c - sum over the faces with u > 0 of u (L_c - L_nbr);
//   adjoint_finish  one thread per cell, in double: lambda_e^n, lambda_m^n
//        (lambda_v = -(sum n lambda_Gamma) / c enters through v = m / rho)
//        and the opacity gradients, scattered to the caller's order.
// The per-cell FP64 work thus runs in kernels of full warps, and the
// per-angle arithmetic in the state precision (GB300's FP64 rate is a small
// fraction of its FP32 rate).
#include <cuda_runtime.h>

#include "rt_internal.cuh"
#include "rt_step_common.cuh"
#include "rt_step_tile.cuh"

namespace rt {
namespace {

using step::positive;
using step::rcp;

constexpr int kThreads = 256;  // threads per block of adjoint_prep / adjoint_finish

// Per-cell record of adjoint_prep (16 values in the state precision): the
// inputs of the per-angle phases and of the per-cell chain.
template <typename R> struct alignas(4 * sizeof(R)) AdjCell {
  R bx, by, bz;  // v / c
  R X;           // interior: x / Gamma = dt cbar (rho kJ + rho kS); emitter: dt cbar (rho kappa)_src
  R f;           // boundary: 1 - min(dt / tau, 1); emitter: I_src
  R cle, lmx, lmy, lmz;  // c lambda_e, lambda_m of step n + 1
  R Tn;          // gas temperature before the step, e_int / (rho c_v)
  R rho, ir, rcv, kP, kJ, kS;  // rho, 1 / rho, rho c_v, opacities per unit mass
};
// Per-cell record of source_reverse_tile for adjoint_finish (8 values in the
// state precision).
template <typename R> struct alignas(4 * sizeof(R)) AdjOut {
  R dle;         // lambda_e^n - lambda_e^{n+1} (= -lambda of the kinetic energy)
  R gP, gJ;      // the per-cell chain's kappa_P, kappa_J gradients
  R gJx;         // sum_a Gamma_a lambda_x_a (the x_a = dt cbar rho (kJ + kS) Gamma_a term)
  R lvx, lvy, lvz;  // sum_a n_a lambda_Gamma_a (emitter: n dI'/dGamma lambda_I')
  R pad;
};

template <typename R> struct AdjArgs {
  int64_t n;
  int A, H, quad_end;
  const R *inv_vol;    // [N]
  const GasStatic *gs; // [N]
  const uint8_t *kind; // [N]
  const double2 *aux;  // [N] (tau or emit_rate, I_src)
  const int64_t *cell_of;  // [N] internal -> caller cell
  const R *dir;        // [A][4] (x, y, z, 0), caller angle order
  const R *wt2;        // [A/2][2] weights of the pairs (p, p + A/2)
  const R *Is;         // [N][A] I* (the transported rows)
  const R *lI1;        // [N][A] lambda_I^{n+1}
  R *Ls;               // [N][A] out: dt/V lambda_I*
  AdjCell<R> *rec;     // [N] adjoint_prep -> source_reverse_tile
  AdjOut<R> *out;      // [N] source_reverse_tile -> adjoint_finish
  double *eint;        // [N] e_int in double (the double chain of float states)
  // caller order: e, m, lambda_e^{n+1}, lambda_m^{n+1} in; lambda_e^n,
  // lambda_m^n out (may alias le1 / lm1: each is read before its cell is
  // written, by the same thread); gP, gJ accumulate
  const double *e, *m, *le1, *lm1;  // [N], [N][3], [N], [N][3]
  double *le, *lm, *gP, *gJ;        // [N], [N][3], [N], [N]
  double dt, cbar, c, a_rad, inv_c;
  R dt_r, k_ex_r;      // dt; 4 pi / cbar
  int newton_max_iter;
};

// 1 / v: float by the approximate reciprocal (v = Gamma or 1 + x Gamma,
// normal or +inf); double refined from it (rcp divides outside float range,
// +inf included).
__device__ __forceinline__ float rcp_pos(float v) { return rcp(v); }
__device__ __forceinline__ double rcp_pos(double v) { return rcp(v); }

// Comoving quantities of one angle of an interior cell: Gamma = 1 - v.n/c,
// w^ = w / Gamma^2, r = 1 / (1 + x), x = X Gamma, I~ = Gamma^4 I*.
template <typename R> struct Ang {
  R G, iG, iG4, wh, r, It;
};
template <typename R> __device__ __forceinline__ Ang<R> comoving_g(R G, R wt, R X, R is) {
  Ang<R> g;
  g.G = G;
  const R xp = fma(X, g.G, R(1));  // 1 + x
  if constexpr (sizeof(R) == 8) {
    // double: one reciprocal of Gamma (1 + x) serves both (the FP64 pipe
    // bounds the double kernel)
    const R p = rcp_pos(g.G * xp);
    g.iG = xp * p;
    g.r = g.G * p;
  } else {
    g.iG = rcp_pos(g.G);
    g.r = rcp_pos(xp);
  }
  const R iG2 = g.iG * g.iG, G2 = g.G * g.G;
  g.iG4 = iG2 * iG2;
  g.wh = wt * iG2;
  g.It = G2 * G2 * is;
  return g;
}
// Sums of phase 1 (unnormalised by N_w = sum w^).
template <typename R> struct CellSums {
  R Nw, SI, SG, S1, lq;
};

// adjoint_prep: the record of internal cell i (caller cell cell_of[i]).
template <typename R> __global__ void adjoint_prep(const AdjArgs<R> a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t c = a.cell_of[i];
  const int kind = a.kind[i];
  const GasStatic gs = a.gs[i];
  const double mx = a.m[3 * c], my = a.m[3 * c + 1], mz = a.m[3 * c + 2];
  const double vc = gs.inv_rho * a.inv_c;
  AdjCell<R> o;
  o.bx = R(mx * vc);
  o.by = R(my * vc);
  o.bz = R(mz * vc);
  o.cle = R(a.c * a.le1[c]);
  o.lmx = R(a.lm1[3 * c]);
  o.lmy = R(a.lm1[3 * c + 1]);
  o.lmz = R(a.lm1[3 * c + 2]);
  o.X = R(a.dt * a.cbar * (gs.rkJ + gs.rkS));
  o.f = R(0);
  if (kind == RT_CELL_BOUNDARY) {
    const double2 ax = a.aux[i];
    o.f = R(1.0 - ((ax.x <= a.dt) ? 1.0 : a.dt / ax.x));
  } else if (kind == RT_CELL_EMITTER) {
    const double2 ax = a.aux[i];
    o.X = R(a.dt * a.cbar * ax.x);
    o.f = R(ax.y);
  }
  const double eint = a.e[c] - 0.5 * (mx * mx + my * my + mz * mz) * gs.inv_rho;
  o.rho = R(gs.rho);
  o.ir = R(gs.inv_rho);
  o.rcv = R(gs.rcv);
  o.kP = R(gs.rkP) * o.ir;
  o.kJ = R(gs.rkJ) * o.ir;
  o.kS = R(gs.rkS) * o.ir;
  o.Tn = R(eint) * (R(1) / o.rcv);
  a.rec[i] = o;
  a.eint[i] = eint;
}

// Phase 2 for one interior cell in the compute type C: the forward
// per-cell chain (the weights normalised, D = S_1 + dt cbar rho kJ S_G =
// 1 - dt cbar rho kS S_G) and its reverse from lambda_q down to lambda_{S_I},
// lambda_{S_G}.  The quartic is solved from the gas temperature before the
// step.  Float states run it in float (the adjoint linearises at the float
// root; its derivatives move by the root's relative error, ~1e-7) and repeat
// it in double when a result is not finite; double states run it in double.
template <typename C> struct Chain {
  C q, lSI, lSG, swl, iNw, dle, gP, gJ;
};
template <typename C> struct ChainIn {
  C rho, ir, rcv, kP, kJ, kS, Tn;
};
template <typename C> __device__ __forceinline__ C tol_of();
template <> __device__ __forceinline__ float tol_of<float>() { return 1e-7f; }
template <> __device__ __forceinline__ double tol_of<double>() { return 1e-15; }

template <typename R> __device__ __forceinline__ ChainIn<R> chain_in(const AdjCell<R> &r) {
  return ChainIn<R>{r.rho, r.ir, r.rcv, r.kP, r.kJ, r.kS, r.Tn};
}
// The same inputs in double, from the gas record and e_int (as adjoint_prep
// forms them for double states).
__device__ __forceinline__ ChainIn<double> chain_in_double(const GasStatic &gs, double eint) {
  const double ir = gs.inv_rho;
  return ChainIn<double>{gs.rho, ir, gs.rcv, gs.rkP * ir, gs.rkJ * ir, gs.rkS * ir,
                         eint * (1.0 / gs.rcv)};
}

template <typename C, typename R>
__device__ Chain<C> cell_chain(const AdjArgs<R> &a, const ChainIn<C> &in, const CellSums<R> &s) {
  Chain<C> o;
  const C iNw = C(1) / C(s.Nw);
  const C SI = C(s.SI) * iNw, SG = C(s.SG) * iNw, S1 = C(s.S1) * iNw, lq = C(s.lq);
  const C rho = in.rho, rcv = in.rcv, irc = C(1) / rcv;
  const C kP = in.kP, kJ = in.kJ, kS = in.kS;
  const C dcb = C(a.dt * a.cbar) * rho, dcc = C(a.dt * a.c) * rho, a_rad = C(a.a_rad);
  const C pi4 = C(4.0 * kPi);
  const C Tn = in.Tn;
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
  o.gP = gP;
  o.gJ = gJ;
  return o;
}

template <typename C> __device__ __forceinline__ bool chain_finite(const Chain<C> &o) {
  return isfinite(o.q) && isfinite(o.lSI) && isfinite(o.lSG) && isfinite(o.swl) &&
         isfinite(o.iNw) && isfinite(o.dle) && isfinite(o.gP) && isfinite(o.gJ);
}

// Phase 2 of a float state's interior cell, in each of its threads: the
// float chain, or the double one where a float result is not finite.
__device__ __forceinline__ Chain<float> float_chain(const AdjArgs<float> &a, int64_t c,
                                                    const AdjCell<float> &rec,
                                                    const CellSums<float> &s) {
  Chain<float> o = cell_chain<float>(a, chain_in(rec), s);
  if (!chain_finite(o)) {
    const Chain<double> d = cell_chain<double>(a, chain_in_double(a.gs[c], a.eint[c]), s);
    o = Chain<float>{float(d.q), float(d.lSI), float(d.lSG), float(d.swl),
                     float(d.iNw), float(d.dle), float(d.gP), float(d.gJ)};
  }
  return o;
}

// adjoint_finish: lambda_e^n, lambda_m^n and the opacity gradients of
// internal cell i, written to caller cell cell_of[i].  lambda_v =
// -(sum n lambda_Gamma) / c enters lambda_m through v = m / rho; the
// x_a = dt cbar rho (kJ + kS) Gamma_a term gives the kappa_J gradient.
template <typename R> __global__ void adjoint_finish(const AdjArgs<R> a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t c = a.cell_of[i];
  const int kind = a.kind[i];
  const double rho = a.gs[i].rho, inv_rho = a.gs[i].inv_rho;
  const double f = -a.inv_c * inv_rho;
  const AdjOut<R> o = a.out[i];
  const double le1 = a.le1[c];
  double lm[3] = {a.lm1[3 * c], a.lm1[3 * c + 1], a.lm1[3 * c + 2]};
  const double lv[3] = {(double)o.lvx, (double)o.lvy, (double)o.lvz};
  if (kind == RT_CELL_BOUNDARY) {
    a.le[c] = le1;
  } else if (kind == RT_CELL_EMITTER) {
    a.le[c] = le1;
    for (int d = 0; d < 3; ++d) lm[d] = lm[d] + f * lv[d];
  } else {
    const double dle = (double)o.dle, lkin = -dle;
    a.le[c] = le1 + dle;
    a.gP[c] += (double)o.gP;
    a.gJ[c] += (double)o.gJ + a.dt * a.cbar * rho * (double)o.gJx;
    const double mom[3] = {a.m[3 * c], a.m[3 * c + 1], a.m[3 * c + 2]};
    for (int d = 0; d < 3; ++d) lm[d] = (lm[d] + mom[d] * inv_rho * lkin) + f * lv[d];
  }
  for (int d = 0; d < 3; ++d) a.lm[3 * c + d] = lm[d];
}

// ------------------------------------------------------------ the kernel
// The per-angle phases (1 and 3) run on the step kernel's tile mapping: 32
// cells x 8 threads, thread `sub` holding the entries of its pair / quad map
// (angle p and its antipode, whose Gamma is 1 + v.n_p where p's is
// 1 - v.n_p).  A cell's sums reduce over its 8 threads (3 shuffles, by xor,
// so that all 8 hold the same sums bit for bit), the 4 cells of a warp at
// once.

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
                                           const Chain<R> &r, R &gJx, R &lGo) {
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
  __device__ __forceinline__ R ex(int j, bool anti, const AdjCell<R> &ci, R k_ex) const {
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
  constexpr bool kLaneChain = sizeof(R) == 4;  // float: the chain in every thread of the cell
  constexpr int kShared = kLaneChain ? 1 : kRevCells;
  __shared__ CellSums<R> sums[kShared];
  __shared__ Chain<R> rev[kShared];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int lc = threadIdx.x / KT, sub = threadIdx.x % KT;
  const int64_t c0 = (int64_t)blockIdx.x * kRevCells;
  const bool live = c0 + lc < a.n;
  const int64_t c = live ? c0 + lc : a.n - 1;  // dead threads shadow the last cell
  const int np = M::count(a.H, sub);
  const AdjCell<R> ci = a.rec[c];  // the cell's 8 threads read the same record
  const int kind = a.kind[c];
  const R k_ex = a.k_ex_r;  // lambda_I* gets 4 pi w (c lambda_e + n . lambda_m) / cbar
  // ---------------- phase 1: the angular sums and lambda_q
  CellSums<R> cs;
  {
    R Nw = 0, SI = 0, SG = 0, S1 = 0, lq = 0;
    if (kind == RT_CELL_INTERIOR) {
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
    cs = CellSums<R>{group_sum(Nw), group_sum(SI), group_sum(SG), group_sum(S1), group_sum(lq)};
  }

  // ---------------- phase 2: the quartic and the per-cell chain
  Chain<R> r{};
  if constexpr (kLaneChain) {
    if (kind == RT_CELL_INTERIOR) r = float_chain(a, c, ci, cs);
  } else {
    if (sub == 0) sums[lc] = cs;
    __syncthreads();
    const int64_t cl = c0 + lane;
    if (warp == 0 && lane < kRevCells && cl < a.n && a.kind[cl] == RT_CELL_INTERIOR)
      rev[lane] = cell_chain<R>(a, chain_in(a.rec[cl]), sums[lane]);
    __syncthreads();
    if (kind == RT_CELL_INTERIOR) r = rev[lc];
  }

  // ---------------- phase 3: per-angle reverse, lambda_I* (the entries read again: the
  // rows are in L1, and nothing per angle stays live across phase 2)
  {
    const R dtv = a.dt_r * a.inv_vol[c];  // the scale the adjoint transport divides out
    Entries<R, M> E;
    E.load(a, c, sub, np);
    R oa[PPT], ob[PPT];
    R gJx = 0, lvx = 0, lvy = 0, lvz = 0;
    if (kind == RT_CELL_BOUNDARY) {
      const R f = dtv * ci.f;
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        oa[j] = f * E.la[j];
        ob[j] = f * E.lb[j];
      }
    } else if (kind == RT_CELL_EMITTER) {
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
    // the cell's record for adjoint_finish: thread `sub` writes value `sub`
    if (live) {
      const R v[8] = {r.dle, r.gP, r.gJ, gJx, lvx, lvy, lvz, R(0)};
      R w = v[0];
#pragma unroll
      for (int k = 1; k < 8; ++k) w = sub == k ? v[k] : w;
      reinterpret_cast<R *>(a.out + c)[sub] = w;
    }
  }
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

template <typename R>
cudaError_t run_adjoint(rt_state *s, const R *I_int, const R *lI1_int, R *lI_int, double dt,
                        const double *e, const double *m, const double *le1, const double *lm1,
                        double *le, double *lm, double *gP, double *gJ) {
  const int64_t N = s->n_cells;
  const int A = s->n_angles;
  const unsigned g1 = (unsigned)((N + kThreads - 1) / kThreads);
  R *Is = reinterpret_cast<R *>(s->d_adj[0]);
  R *Ls = reinterpret_cast<R *>(s->d_adj[1]);
  char *ws = reinterpret_cast<char *>(s->d_adj_ws);  // [N] records, [N] results, [N] e_int
  AdjArgs<R> a;
  a.n = N;
  a.A = A;
  a.H = A / 2;
  a.quad_end = s->quad_end;
  a.inv_vol = reinterpret_cast<const R *>(s->d_inv_vol);
  a.gs = s->d_gs;
  a.kind = s->d_kind;
  a.aux = s->d_aux;
  a.cell_of = s->d_cell_of;
  a.dir = reinterpret_cast<const R *>(s->d_dir);
  a.wt2 = reinterpret_cast<const R *>(s->d_wt);
  a.Is = Is;
  a.lI1 = lI1_int;
  a.Ls = Ls;
  a.rec = reinterpret_cast<AdjCell<R> *>(ws);
  a.out = reinterpret_cast<AdjOut<R> *>(ws + sizeof(AdjCell<R>) * (size_t)N);
  a.eint = reinterpret_cast<double *>(ws + (sizeof(AdjCell<R>) + sizeof(AdjOut<R>)) * (size_t)N);
  a.e = e;
  a.m = m;
  a.le1 = le1;
  a.lm1 = lm1;
  a.le = le;
  a.lm = lm;
  a.gP = gP;
  a.gJ = gJ;
  a.dt = dt;
  a.cbar = s->params.cbar;
  a.c = s->params.c;
  a.a_rad = s->params.a_rad;
  a.inv_c = 1.0 / s->params.c;
  a.dt_r = R(dt);
  a.k_ex_r = R(4.0 * kPi / s->params.cbar);
  a.newton_max_iter = s->params.newton_max_iter;
  adjoint_prep<R><<<g1, kThreads, 0, s->stream>>>(a);
  s->launches++;
  cudaError_t err = launch_transport(s, dt, I_int, Is, false);
  if (err != cudaSuccess) return err;
  launch_reverse<R>(s, a);
  s->launches++;
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  err = launch_transport(s, dt, Ls, lI_int, true);
  if (err != cudaSuccess) return err;
  adjoint_finish<R><<<g1, kThreads, 0, s->stream>>>(a);
  s->launches++;
  return cudaGetLastError();
}

}  // namespace

cudaError_t adjoint_step(rt_state *s, double dt, const void *I, const double *e, const double *m,
                         const void *lI1, const double *le1, const double *lm1, void *lI,
                         double *le, double *lm, double *gP, double *gJ) {
  // per-cell arrays are device pointers in the caller's order (adjoint_prep
  // gathers, adjoint_finish scatters); the rows are permuted into dense
  // internal rows (stride A) and back
  void *I_int = s->d_adj[2], *lI1_int = s->d_adj[3], *lI_int = s->d_adj[4];
  cudaError_t err = launch_permute_in(s, I, I_int, s->n_angles);
  if (err == cudaSuccess) err = launch_permute_in(s, lI1, lI1_int, s->n_angles);
  if (err != cudaSuccess) return err;
  if (s->precision == RT_FP32)
    err = run_adjoint<float>(s, (const float *)I_int, (const float *)lI1_int, (float *)lI_int, dt,
                             e, m, le1, lm1, le, lm, gP, gJ);
  else
    err = run_adjoint<double>(s, (const double *)I_int, (const double *)lI1_int,
                              (double *)lI_int, dt, e, m, le1, lm1, le, lm, gP, gJ);
  if (err != cudaSuccess) return err;
  return launch_permute_out(s, lI_int, lI, s->n_angles);
}

}  // namespace rt
