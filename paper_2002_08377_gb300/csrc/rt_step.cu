// Fused radiation step: upwind transport (Sec. 2.2) + implicit comoving
// source update with gas exchange (Sec. 2.3), boundary cells (Sec. 2.4) and
// emitter cells (Sec. 2.5), one kernel per step.
//
// Layout: the intensity row of a cell stores the A/2 antipodal pairs
// (angle p, angle p + A/2) side by side.  The flux coefficient of the
// antipode through a face is u(p + A/2) = -(n_p . s) - w, so one dot product
// serves both angles; on a static mesh exactly one of the two is inflow.
//
// Block = 32 cells x 8 threads.  Which pairs a thread owns is a policy:
//   PairMap  thread `sub` owns pairs sub + 8 j (j < PPT), one 8-byte (float)
//            or 16-byte (double) access each -- any A;
//   QuadMap  float rows with A a multiple of 16: thread `sub` owns the pair
//            quads sub + 8 i (one 16-byte access each, so a cell's 8 threads
//            read 128 contiguous bytes of a neighbour row per instruction)
//            and, when A/2 is not a multiple of 16, the pair 16 Q4 + sub.
// The neighbour-row gathers of the face loop are bound by the L1 data pipe
// (one wavefront per cache line an instruction touches), so wider per-thread
// accesses cut the face loop's cost directly.  The float kernel with QuadMap
// also copies the block's face slots and neighbour indices into shared
// memory at its start.  Registers are capped so that 1024 threads share an
// SM (768 for more than 5 pairs per thread).
// Phases:
//   A  all threads: transport over the cell's faces in slot order (no
//      atomics, deterministic), comoving weights and the angular sums of
//      Eq. (Jcom); each cell's 8 lanes reduce with shuffles;
//   B  the gas temperature quartic, between two block barriers: double
//      states solve it in double with one lane per cell in the first
//      CPB / 32 warps; float states find the float root in all 8 lanes of
//      the cell and one lane per cell refines it by Newton in double (with
//      float_quartic = 1 the float root is final: no barrier);
//   C  all threads: new intensities, store, radiation change per cell;
//   D  after a block barrier, one lane per cell (first CPB / 32 warps): gas energy /
//      momentum (or tally) update in double (Eqs. gas1, gas2).
// The double-precision work is lane-per-cell because GB300's FP64 rate is a
// small fraction of its FP32 rate.
#include <cuda_runtime.h>

#include "rt_internal.cuh"
#include "rt_step_common.cuh"
#include "rt_step_tile.cuh"

namespace rt {
namespace {
using namespace step;

// Per-block sums exchanged between the phases.
template <typename R> struct Shared {
  R sI[CPB], sG[CPB], s1[CPB];  // the sums of Eq. (Jcom) and sum w~/(1+x), unnormalised
  R q[CPB];                     // dt cbar rho (kP B + kS J) per interior cell
  float qa[CPB], qg[CPB], qT[CPB];  // float states: alpha, g and the float temperature root
  R dE[CPB], dF[3][CPB];        // sum w (I* - I') and sum w n (I* - I')
  unsigned bad[CPB];
};

// The Lorentz factor in Gamma = gamma (1 -+ v.n / c) (Sec. 2.3) of a cell
// with v / c = (bx, by, bz): 1 for the first-order transformation, else
// (1 - v^2 / c^2)^(-1/2).
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
template <typename R> __device__ __forceinline__ R frame_gamma(int boost, R bx, R by, R bz) {
  return boost ? rsqrt_r(R(1) - fma(bx, bx, fma(by, by, bz * bz))) : R(1);
}

// Temperature quartic of one interior cell and its emission term
// q = dt cbar rho (kP B + kS J~).  With w~ normalised, x_a = dt cbar rho
// (kJ + kS) Gamma_a and the sums S_I, S_G of Eq. (Jcom), S_1 = sum w~ / (1 + x):
//   D = 1 - dt cbar rho kS S_G = S_1 + dt cbar rho kJ S_G,
//   1 - dt cbar rho kJ S_G / D = S_1 / D,
// so the quartic alpha T^4 + rho c_v T = g of Eq. (com rad thermal disc) has
// alpha = dt c a rho kP S_1 / D and g = (e - kinetic) + dt c 4 pi rho kJ S_I / D:
// sums of positive terms, no cancellation when x >> 1.  The weight
// normalisation cancels in every ratio.  Sets status bits in `bad`.
template <typename R>
__device__ __forceinline__ double source_q(const StepArgs<R> &a, const GasStatic &g,
                                           const GasDyn &d, double SI, double SG, double S1,
                                           unsigned &bad) {
  const double dJ = a.k_dcr * g.rkJ, dP = a.k_dcr * g.rkP, dS = a.k_dcr * g.rkS;
  const double rU = rcp(fma(dJ, SG, S1));
  const double kin = 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * g.inv_rho;
  const double alpha = a.k_alpha * g.rkP * S1 * rU;
  const double eint = d.e - kin;
  const double gq = eint + a.k_g * g.rkJ * SI * rU;
  double T = 0.0, dPT = dP;  // dPT: dP with kappa_P at T^{n+1}
  if (!(gq >= 0.0) || !(alpha >= 0.0)) {
    bad |= ST_NONFINITE;
  } else if (a.beta_P == 0.0) {
    if (quartic_root(alpha, g.rcv, gq, eint / g.rcv, 1e-15, a.newton_max_iter, &T))
      bad |= ST_NONCONV;
  } else {
    // kappa_P (T/T_ref)^beta_P T^4 = kappa_P T_ref^-beta_P T^(4 + beta_P)
    if (power_root(alpha * a.tref_mbP, 4.0 + a.beta_P, g.rcv, gq, eint / g.rcv, 1e-15,
                   a.newton_max_iter, &T))
      bad |= ST_NONCONV;
    dPT = dP * pow(T / a.T_ref, a.beta_P);
  }
  const double B = a.a_rad * (T * T) * (T * T) * (1.0 / (4.0 * kPi));
  const double J = fma(dPT * B, SG, SI) * rU;  // the J~ of Eq. (Jcom)
  return fma(dPT, B, dS * J);
}

// The temperature equation of a float state's cell in float: the
// coefficients of source_q from the float copies of the cell's opacities and
// the float angular sums (alpha multiplies T^(4 + beta_P) T_ref^-beta_P),
// with rU = 1 / D and dP, dS = dt cbar rho kappa_P, kappa_s.
struct QuarticF {
  float alpha, gq, rU, dP, dS;
};
__device__ __forceinline__ QuarticF float_coeffs(const StepArgs<float> &a, float rkP, float rkJ,
                                                 float rkS, float eint, float SI, float SG,
                                                 float S1) {
  QuarticF k;
  const float dJ = a.k_dcr_f * rkJ;
  k.dP = a.k_dcr_f * rkP;
  k.dS = a.k_dcr_f * rkS;
  k.rU = rcp(fmaf(dJ, SG, S1));
  k.alpha = a.k_alpha_f * rkP * S1 * k.rU;
  k.gq = eint + a.k_g_f * rkJ * SI * k.rU;
  if (a.beta_P_f != 0.0f) k.alpha *= a.tref_mbP_f;
  return k;
}
// Float root of the cell's equation from the pre-step temperature (returns
// 1 if Newton did not converge).
__device__ __forceinline__ int float_root(const StepArgs<float> &a, const QuarticF &k, float rcv,
                                          float eint, float *T) {
  if (a.beta_P_f == 0.0f)
    return quartic_root(k.alpha, rcv, k.gq, eint * rcp(rcv), 1e-7f, a.newton_max_iter, T);
  return power_root(k.alpha, 4.0f + a.beta_P_f, rcv, k.gq, eint * rcp(rcv), 1e-7f,
                    a.newton_max_iter, T);
}
// The emission term q = dt cbar rho (kP(T) B(T) + kS J~) in float.
__device__ __forceinline__ float float_q(const StepArgs<float> &a, const QuarticF &k, float T,
                                         float SI, float SG) {
  float dPT = k.dP;  // dP with kappa_P at T^{n+1}
  if (a.beta_P_f != 0.0f) dPT = k.dP * powf(T / a.T_ref_f, a.beta_P_f);
  const float B = a.a_rad_4pi_f * (T * T) * (T * T);
  const float J = fmaf(dPT * B, SG, SI) * k.rU;
  return fmaf(dPT, B, k.dS * J);
}

// The same as source_q in float for float states (float_quartic = 1), from
// the float coefficients and the internal energy e - rho v^2 / 2 that the
// previous gas update left in cellv; coefficients or an emission term
// outside float range fall back to the double solve.
__device__ __forceinline__ float source_q_float(const StepArgs<float> &a, int64_t c, float rkP,
                                                float rkJ, float rkS, float rcv, float eint,
                                                float SI, float SG, float S1, unsigned &bad) {
  const QuarticF k = float_coeffs(a, rkP, rkJ, rkS, eint, SI, SG, S1);
  if (!(k.gq >= 0.0f) || !(k.alpha >= 0.0f)) {
    bad |= ST_NONFINITE;
    return 0.0f;
  }
  if (isfinite(k.alpha) && isfinite(k.gq)) {
    float T;
    const int nc = float_root(a, k, rcv, eint, &T);
    const float q = float_q(a, k, T, SI, SG);
    if (isfinite(q)) {
      if (nc) bad |= ST_NONCONV;
      return q;
    }
  }
  return (float)source_q(a, a.gs[c], a.gd[c], (double)SI, (double)SG, (double)S1, bad);
}

// q of an interior cell of a float state (float_quartic = 0), one lane per
// cell: the float coefficients and root as in source_q_float, the root
// refined in double by refine_root, q in float from it; where a float value
// is not finite or the float Newton did not converge, the double solve of
// source_q.
__device__ __forceinline__ float source_q_refined(const StepArgs<float> &a, const GasStatic &gr,
                                                  const GasDyn &gd, float SI, float SG, float S1,
                                                  float eint, unsigned &bad) {
  const QuarticF k = float_coeffs(a, gr.frkP, gr.frkJ, gr.frkS, eint, SI, SG, S1);
  if (!(k.gq >= 0.0f) || !(k.alpha >= 0.0f)) {
    bad |= ST_NONFINITE;
    return 0.0f;
  }
  float Tf;
  if (isfinite(k.alpha) && isfinite(k.gq) && !float_root(a, k, gr.frcv, eint, &Tf) &&
      isfinite(Tf)) {
    const double T = refine_root(k.alpha, a.beta_P_f, a.beta_P, gr.rcv, k.gq, Tf);
    const float q = float_q(a, k, (float)T, SI, SG);
    if (isfinite(q)) return q;
  }
  return (float)source_q(a, gr, gd, (double)SI, (double)SG, (double)S1, bad);
}

// One block of CPB cells: phases A-D (see the top of the file).  STAGED:
// the caller has started the copies of the tile's slots and gas records into
// `stage`, and the face loop waits for them; otherwise slots are read from
// global memory and the lane-per-cell threads copy the gas records into
// `gas` themselves.
// How float states solve the temperature equation (phase B): chosen at run
// time from StepArgs::float_quartic, or fixed by the kernel instantiation.
enum : int { QM_RUNTIME = 0, QM_FLOAT = 1, QM_REFINE = 2 };

template <typename R, typename M, bool MOVING, bool STAGED, int QM = QM_RUNTIME>
__device__ __forceinline__ void tile_step(const StepArgs<R> &a, const int64_t tile, Shared<R> &sh,
                                          SharedGas *gas, const StageView &stage) {
  using V = pair_t<R>;
  constexpr int PPT = M::PPT;
  const int lc = threadIdx.x / KT;
  const int sub = threadIdx.x % KT;
  const int64_t cell = tile * CPB + lc;
  const bool live = cell < a.n_cells;
  const int64_t c = live ? cell : a.n_cells - 1;  // dead lanes shadow the last cell
  const int RS = a.row;  // reals between intensity rows
  const int np = M::count(a.half, sub);

  // lane-per-cell phases: thread t < CPB (the first CPB / 32 warps) takes cell t
  const int lp = threadIdx.x;
  const bool lpc = lp < CPB;
  const int64_t cl = tile * CPB + lp;
  if (!STAGED && lpc && cl < a.n_cells) {
    // prefetch of the cells' gas state for phases B and D
    const char *g = reinterpret_cast<const char *>(a.gs + cl);
    const char *d = reinterpret_cast<const char *>(a.gd + cl);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      cp_async16(reinterpret_cast<char *>(&gas->gs[lp]) + 16 * k, g + 16 * k);
#pragma unroll
    for (int k = 0; k < 2; ++k)
      cp_async16(reinterpret_cast<char *>(&gas->gd[lp]) + 16 * k, d + 16 * k);
  }

  // ---------------- phase A: transport, I* = I - dt/V sum_f u I_up
  R nx[PPT], ny[PPT], nz[PPT], Ia[PPT], Ib[PPT], acca[PPT], accb[PPT];
  M::load(a.I_in + (size_t)c * RS, sub, Ia, Ib, np);
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    load_dir(a.dir, (M::FULL || j < np) ? M::pair(j, sub) : 0, nx[j], ny[j], nz[j]);
    acca[j] = R(0);
    accb[j] = R(0);
  }
  if constexpr (STAGED) {
    const int64_t kb = a.ptr[tile * CPB];
    const int k0 = (int)(a.ptr[c] - kb), k1 = (int)(a.ptr[c + 1] - kb);
    cp_async_wait_all();
    __syncthreads();  // the block's stage has landed
    if (!a.src_only)
      face_sum<R, M, MOVING, !MOVING, TRANSPORT_FORWARD>(
          reinterpret_cast<const typename SlotOf<R>::type *>(stage.slot), stage.nbr, a.wface,
          a.uface, a.half, k0, k1, a.I_in, RS, sub, nx, ny, nz, Ia, Ib, acca, accb, np);
  } else {
    if (!a.src_only)
      face_sum<R, M, MOVING, false, TRANSPORT_FORWARD>(a.slot, a.nbr, a.wface, a.uface, a.half, a.ptr[c],
                                    a.ptr[c + 1], a.I_in, RS, sub, nx, ny, nz, Ia, Ib, acca, accb,
                                    np);
  }
  {
    const R dtv = a.dt_r * a.inv_vol[c];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      Ia[j] = fma(-dtv, acca[j], Ia[j]);  // I*
      Ib[j] = fma(-dtv, accb[j], Ib[j]);
    }
    if constexpr (MOVING) {
      // geometric conservation law (volumes change only on a moving mesh):
      // V^{n+1} I* = V^n I - dt sum_f u I_up, i.e. the fixed-volume I* times
      // V^n / V^{n+1} = 1 / (1 + dt rate / V^n)
      if (a.gcl_rate && !a.src_only) {
        const R ratio = rcp(fma(dtv, R(a.gcl_rate[c]), R(1)));
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          Ia[j] *= ratio;
          Ib[j] *= ratio;
        }
      }
    }
  }

  // comoving frame (first order in v/c): Gamma = 1 -+ v.n / c, and the
  // angular sums of Eq. (Jcom): w~ = w / Gamma^2 (normalised by their sum),
  // S_I = sum w~ Gamma^4 I* / (1 + x Gamma), S_G = sum w~ Gamma / (1 + x Gamma).
  // To all orders Gamma = gamma G with G = 1 -+ v.n / c: the weights'
  // normalisation cancels gamma^2, so gamma enters only per cell -- x = (xs
  // gamma) G, S_I -> gamma^4 S_I, S_G -> gamma S_G (S_1 unchanged) and, in
  // phase C, q -> q / gamma^3 (emitters: rate gamma, source / gamma^4).
  // With gamma = 1 these scalings are exact.
  const int kind = a.kind[c];
  const R icr = a.inv_c_r;
  const R vxc = a.cellv[4 * c] * icr, vyc = a.cellv[4 * c + 1] * icr,
          vzc = a.cellv[4 * c + 2] * icr;
  R xs, eint = a.cellv[4 * c + 3];  // dt cbar rho (kJ + kS), internal energy
  R fkP = 0, fkJ = 0, fkS = 0, fcv = 0;
  if constexpr (sizeof(R) == 4) {
    const float4 gf = __ldg(reinterpret_cast<const float4 *>(&a.gs[c].frkP));
    fkP = gf.x;
    fkJ = gf.y;
    fkS = gf.z;
    fcv = gf.w;
    xs = a.dt_cbar_r * (fkJ + fkS);
  } else {
    xs = a.dt_cbar_r * R(a.gs[c].rkJ + a.gs[c].rkS);
  }
  if (a.boost) xs *= frame_gamma(a.boost, vxc, vyc, vzc);
  const V *W2 = reinterpret_cast<const V *>(a.wt2);  // (w_p, w_{p+H})
  const V one = mk(R(1), R(1)), XS = mk(xs, xs);
  // Gamma = (1 - bn, 1 + bn) for the pair, bn = v . n_p / c; the directions
  // are read again in phase C rather than held across phase B
  V sIv = mk(R(0), R(0)), sGv = sIv, s1v = sIv;  // unnormalised: cancels in phase B
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    if (M::FULL || j < np) {
      // t = w / (Gamma^2 (1 + x Gamma)): one reciprocal per angle
      const R bn = fma(vxc, nx[j], fma(vyc, ny[j], vzc * nz[j]));
      const V G = mk(R(1) - bn, R(1) + bn);
      const V G2 = pmul(G, G);
      const V t = pmul(W2[M::pair(j, sub)], prcp<R>(pmul(G2, pfma(XS, G, one))));
      s1v = padd(s1v, t);
      sIv = pfma(pmul(t, pmul(G2, G2)), mk(Ia[j], Ib[j]), sIv);
      sGv = pfma(t, G, sGv);
    }
  }
  R sI = sIv.x + sIv.y, sG = sGv.x + sGv.y, s1 = s1v.x + s1v.y;
  sI = cell_sum(sI);
  sG = cell_sum(sG);
  s1 = cell_sum(s1);
  if (a.boost) {
    const R g = frame_gamma(a.boost, vxc, vyc, vzc), g2 = g * g;
    sI *= g2 * g2;
    sG *= g;
  }

  // ---------------- phase B: temperature quartic
  R q = 0;           // dt cbar rho (kP B + kS J~) of an interior cell
  unsigned bad = 0;  // status bits of the cell
  const GasStatic *gs_s = STAGED ? stage.gas->gs : gas->gs;
  const GasDyn *gd_s = STAGED ? stage.gas->gd : gas->gd;
  bool lane_solve = false;  // float states with float_quartic: in float, in every lane
  if constexpr (sizeof(R) == 4)
    lane_solve = QM == QM_FLOAT || (QM == QM_RUNTIME && a.float_quartic != 0);
  if (lane_solve) {
    // every lane of the cell solves the cell's quartic in float (the sums
    // are already in all 8 lanes), no block barrier
    if constexpr (sizeof(R) == 4)
      if (kind == RT_CELL_INTERIOR)
        q = source_q_float(a, c, fkP, fkJ, fkS, fcv, eint, sI, sG, s1, bad);
  } else if constexpr (sizeof(R) == 4 && QM == QM_REFINE) {
    // float states (default, staged kernels): every lane of the cell finds
    // the float root from the float coefficients (no barrier); one lane per
    // cell then refines it by Newton in double (the FP64 temperature solve)
    // and forms q, or, where the float solve failed, runs the whole double
    // solve of source_q
    float Tf = 0.0f;
    unsigned fst = 0;  // 0: float root, 1: solve in double, 2: non-finite coefficients
    float qa = 0.0f, qg = 0.0f;
    if (kind == RT_CELL_INTERIOR) {
      const QuarticF kc = float_coeffs(a, fkP, fkJ, fkS, eint, sI, sG, s1);
      qa = kc.alpha;
      qg = kc.gq;
      if (!(qg >= 0.0f) || !(qa >= 0.0f))
        fst = 2;
      else if (!isfinite(qa) || !isfinite(qg) || float_root(a, kc, fcv, eint, &Tf) ||
               !isfinite(Tf))
        fst = 1;
    }
    if (sub == 0) {
      sh.sI[lc] = sI;
      sh.sG[lc] = sG;
      sh.s1[lc] = s1;
      sh.qa[lc] = qa;
      sh.qg[lc] = qg;
      sh.qT[lc] = Tf;
      sh.bad[lc] = fst;
    }
    __syncthreads();
    // the double step: lanes 0-15 of warps 0 and 1, one cell each (measured
    // 2 % faster per step than the 32 lanes of warp 0, 3 % faster than four
    // lanes of each of the eight warps)
    const int rp = (threadIdx.x >> 5) * 16 + (threadIdx.x & 31);
    const int64_t rc = tile * CPB + rp;
    if ((threadIdx.x & 31) < 16 && rp < CPB) {
      float ql = 0.0f;
      unsigned bl = 0;
      if (rc < a.n_cells && a.kind[rc] == RT_CELL_INTERIOR) {
        const unsigned st = sh.bad[rp];
        const GasStatic &gr = gs_s[rp];
        if (st == 0) {
          const double T = refine_root(sh.qa[rp], a.beta_P_f, a.beta_P, gr.rcv, sh.qg[rp],
                                       sh.qT[rp]);
          const QuarticF k = float_coeffs(a, gr.frkP, gr.frkJ, gr.frkS, 0.0f, sh.sI[rp],
                                          sh.sG[rp], sh.s1[rp]);
          ql = float_q(a, k, (float)T, sh.sI[rp], sh.sG[rp]);
        }
        if (st == 2) {
          bl = ST_NONFINITE;
        } else if (st == 1 || !isfinite(ql)) {
          ql = (float)source_q(a, gr, gd_s[rp], (double)sh.sI[rp], (double)sh.sG[rp],
                               (double)sh.s1[rp], bl);
        }
      }
      sh.q[rp] = ql;
      sh.bad[rp] = bl;
    }
    __syncthreads();
    q = sh.q[lc];
    bad = sh.bad[lc];
  } else if constexpr (sizeof(R) == 4) {
    // float states (default, pair-map kernels): one lane per cell finds the float root from
    // the float coefficients, refines it by Newton in double (the FP64
    // temperature solve) and forms q from it; where the float solve fails it
    // runs the whole double solve of source_q
    if (sub == 0) {
      sh.sI[lc] = sI;
      sh.sG[lc] = sG;
      sh.s1[lc] = s1;
    }
    if (!STAGED && lpc) cp_async_wait_all();
    __syncthreads();
    if (lpc) {
      float ql = 0.0f;
      unsigned bl = 0;
      if (cl < a.n_cells && a.kind[cl] == RT_CELL_INTERIOR)
        ql = source_q_refined(a, gs_s[lp], gd_s[lp], sh.sI[lp], sh.sG[lp], sh.s1[lp],
                              a.cellv[4 * cl + 3], bl);
      sh.q[lp] = ql;
      sh.bad[lp] = bl;
    }
    __syncthreads();
    q = sh.q[lc];
    bad = sh.bad[lc];
  } else {
    // double states: the quartic in double, one lane per cell, so the FP64
    // work is issued by one warp for 32 cells
    if (sub == 0) {
      sh.sI[lc] = sI;
      sh.sG[lc] = sG;
      sh.s1[lc] = s1;
    }
    if (!STAGED && lpc) cp_async_wait_all();
    __syncthreads();
    if (lpc) {
      R ql = 0;
      unsigned bl = 0;
      if (cl < a.n_cells && a.kind[cl] == RT_CELL_INTERIOR)
        ql = R(source_q(a, gs_s[lp], gd_s[lp], (double)sh.sI[lp], (double)sh.sG[lp],
                        (double)sh.s1[lp], bl));
      sh.q[lp] = ql;
      sh.bad[lp] = bl;
    }
    __syncthreads();
    q = sh.q[lc];
    bad = sh.bad[lc];
  }

  // ---------------- phase C: new intensities and the radiation change
  R de = 0, dfx = 0, dfy = 0, dfz = 0;
  unsigned nonfinite = 0;
  {
    // boundary: I' = I* - (I* - I0) f; interior: I~' = (I~ + q Gamma) / (1 + x Gamma),
    // i.e. I' = (I* + q / Gamma^3) / (1 + x Gamma); emitter: the same with
    // x -> dt cbar (rho kappa)_src and q -> that rate times I_src (Sec. 2.5).
    // The radiation change I* - I' that the gas receives: float states take
    // the difference of the stored intensities (the energy bookkeeping is
    // then exact in float); double states take the source term itself,
    // (I* Gamma^3 x Gamma - q) / (Gamma^3 (1 + x Gamma)) and f (I* - I0),
    // whose rounding is relative to the change, not to I* (optically thin
    // cells change I by a small fraction per step).
    R na[PPT], nb[PPT];
    constexpr int ND = sizeof(R) == 8 ? PPT : 1;
    R da[ND], db[ND];  // double states: the change I* - I'
    if (kind == RT_CELL_BOUNDARY) {
      const double2 ax = a.aux[c];
      const R f = R((ax.x <= a.dt) ? 1.0 : a.dt / ax.x);
      R tx[PPT], ty[PPT];
      M::load(a.I0 + (size_t)a.bc_row[c] * RS, sub, tx, ty, np);
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        na[j] = fma(-f, Ia[j] - tx[j], Ia[j]);
        nb[j] = fma(-f, Ib[j] - ty[j], Ib[j]);
        if constexpr (sizeof(R) == 8) {
          da[j] = f * (Ia[j] - tx[j]);
          db[j] = f * (Ib[j] - ty[j]);
        }
      }
    } else {
      R qq, xx = xs;
      if (kind == RT_CELL_EMITTER) {
        const double2 ax = a.aux[c];
        xx = R(a.dt * a.cbar * ax.x);
        qq = xx * R(ax.y);
        if (a.boost) {
          const R g = frame_gamma(a.boost, vxc, vyc, vzc), g2 = g * g;
          xx *= g;
          qq = xx * R(ax.y) / (g2 * g2);
        }
      } else {
        qq = q;
        if (a.boost) {
          const R g = frame_gamma(a.boost, vxc, vyc, vzc);
          qq = q / (g * g * g);
        }
      }
      const V XX = mk(xx, xx), QQ = mk(qq, qq);
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        // I' = (I* Gamma^3 + q) / (Gamma^3 (1 + x Gamma))
        R ux, uy, uz;
        load_dir(a.dir, (M::FULL || j < np) ? M::pair(j, sub) : 0, ux, uy, uz);
        const R bn = fma(vxc, ux, fma(vyc, uy, vzc * uz));
        const V G = mk(R(1) - bn, R(1) + bn);
        const V G3 = pmul(pmul(G, G), G);
        if constexpr (sizeof(R) == 8) {
          const V XG = pmul(XX, G);
          const V r = prcp<R>(pmul(G3, padd(XG, one)));
          const V t = pmul(mk(Ia[j], Ib[j]), G3);
          const V n = pmul(padd(t, QQ), r);
          const V d = pmul(pfma(t, XG, mk(-qq, -qq)), r);
          na[j] = n.x;
          nb[j] = n.y;
          da[j] = d.x;
          db[j] = d.y;
        } else {
          const V n = pmul(pfma(mk(Ia[j], Ib[j]), G3, QQ), prcp<R>(pmul(G3, pfma(XX, G, one))));
          na[j] = n.x;
          nb[j] = n.y;
        }
      }
    }
    if (live) M::store(a.I_out + (size_t)c * RS, sub, na, nb, np);
    V dev = mk(R(0), R(0));
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      if (M::FULL || j < np) {
        const int p = M::pair(j, sub);
        V d;
        if constexpr (sizeof(R) == 8)
          d = pmul(W2[p], mk(da[j], db[j]));
        else
          d = pmul(W2[p], psub(mk(Ia[j], Ib[j]), mk(na[j], nb[j])));
        dev = padd(dev, d);
        const R df = d.x - d.y;  // the antipode has direction -n
        R ux, uy, uz;
        load_dir(a.dir, p, ux, uy, uz);
        dfx = fma(ux, df, dfx);
        dfy = fma(uy, df, dfy);
        dfz = fma(uz, df, dfz);
      }
    }
    de = dev.x + dev.y;
    // a non-finite new intensity makes its weighted change, and so de,
    // non-finite (the weights are positive; the double states' change has
    // the same factors as the intensity)
    if (!isfinite(de)) nonfinite = ST_NONFINITE;
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
    sh.bad[lc] = bad | nonfinite;
  }
  if (sizeof(R) == 4 && !STAGED && lpc) cp_async_wait_all();
  __syncthreads();

  // ---------------- phase D: gas exchange (Eqs. gas1, gas2), one lane per cell
  if (lpc && cl < a.n_cells) {
    // dE_gas = (c/cbar) 4 pi sum w dI, d(rho v) = (4 pi c sum w n dI) / (c cbar)
    const double dE = a.k_fe * (double)sh.dE[lp];
    const double dx = a.k_fm * (double)sh.dF[0][lp], dy = a.k_fm * (double)sh.dF[1][lp],
                 dz = a.k_fm * (double)sh.dF[2][lp];
    if (!a.commit) {
      // stage 1 of the van Leer step: the gas update is discarded
    } else if (a.kind[cl] == RT_CELL_INTERIOR) {
      GasDyn d = gd_s[lp];
      d.e += dE;
      d.mx += dx;
      d.my += dy;
      d.mz += dz;
      a.gd[cl] = d;
      // frame velocity and internal energy for the next step
      const double ir = gs_s[lp].inv_rho;
      const double kin = 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * ir;
      store4(a.cellv + 4 * cl, R(d.mx * ir), R(d.my * ir), R(d.mz * ir), R(d.e - kin));
      if (a.beta_J != 0.0) {
        // kappa_J of the next step, at its starting temperature
        const double rkJ = a.rkJ0[cl] * pow((d.e - kin) / gs_s[lp].rcv / a.T_ref, a.beta_J);
        a.gs_w[cl].rkJ = rkJ;
        a.gs_w[cl].frkJ = (float)rkJ;
      }
    } else {
      double *x = a.ext + 4 * cl;
      x[0] += dE;
      x[1] += dx;
      x[2] += dy;
      x[3] += dz;
    }
    unsigned bad = sh.bad[lp];
    if (MOVING && a.gcl_rate && a.commit) {
      // the cell's volume for the next step, V^{n+1} = V^n + dt sum_f A w . n;
      // this step needed V^n >= dt max_a sum_f max(u, 0) (the float factor
      // carries a ~1e-6 relative error, inside the margin)
      const double V = a.volume[cl];
      if (a.dt * ((double)a.gcl_kv[cl] * a.gcl_kv_unit) > V * (1.0 + 1e-5)) bad |= ST_CFL;
      const double V1 = __dadd_rn(V, __dmul_rn(a.dt, a.gcl_rate[cl]));
      a.volume[cl] = V1;
      a.inv_vol_w[cl] = R(1.0 / V1);
    }
    if (bad) {
      atomicOr(a.status, bad);
      atomicMin(a.bad_cell, (unsigned long long)cl);
    }
  }
}

// Resident threads per SM the register cap aims at: float kernels with up
// to 5 pairs per thread fit 1024 (64 registers), wider ones 768, double 512.
template <typename R, int PPT> constexpr int min_blocks() {
  return (sizeof(R) == 4 ? (PPT <= 5 ? 1024 : 768) : 512) / NT;
}

// One block per CPB cells.
template <typename R, typename M, bool MOVING>
__global__ void __launch_bounds__(NT, min_blocks<R, M::PPT>()) step_kernel(const StepArgs<R> a) {
  __shared__ Shared<R> sh;
  __shared__ SharedGas gas;
  tile_step<R, M, MOVING, false>(a, blockIdx.x, sh, &gas, StageView{});
}

// Float kernel with the QuadMap: the block first starts the copies of its
// slots and gas records into shared memory, then loads its own rows and
// directions while they land (tile_step waits before the face loop).
template <typename M, bool MOVING, int QM>
__global__ void __launch_bounds__(NT, min_blocks<float, M::PPT>())
    step_kernel_staged(const StepArgs<float> a, int cap) {
  __shared__ Shared<float> sh;
  extern __shared__ __align__(128) unsigned char dyn[];
  const StageView v = stage_at(dyn, cap, MOVING);
  issue_stage<MOVING>(a, blockIdx.x, v);
  tile_step<float, M, MOVING, true, QM>(a, blockIdx.x, sh, nullptr, v);
}

// Fills the kernel arguments and launches one step with pair map M.
template <typename R, typename M, bool MOVING, bool STAGED>
cudaError_t launch_t(rt_state *s, double dt, const StepIO &io) {
  StepArgs<R> a;
  a.n_cells = s->n_cells;
  a.n_angles = s->n_angles;
  a.half = s->n_angles / 2;
  a.row = s->row_stride;
  a.ptr = s->d_ptr;
  a.nbr = s->d_nbr;
  a.slot = reinterpret_cast<const typename SlotOf<R>::type *>(s->d_slot);
  a.slot_nb = s->d_slot_nb;
  a.uface = s->d_uface;
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
  a.I_in = reinterpret_cast<const R *>(io.in);
  a.I_out = reinterpret_cast<R *>(io.out);
  a.src_only = io.src_only ? 1 : 0;
  a.commit = io.commit ? 1 : 0;
  a.boost = s->params.boost;
  a.gcl_rate = s->d_gcl_rate;
  a.gcl_kv = s->d_gcl_kv;
  a.gcl_kv_unit = 1.0 / s->screen_scale;
  a.volume = s->d_volume;
  a.inv_vol_w = reinterpret_cast<R *>(s->d_inv_vol);
  a.beta_P = s->params.beta_P;
  a.beta_J = s->params.beta_J;
  a.T_ref = s->params.T_ref;
  a.tref_mbP = a.beta_P != 0.0 ? pow(a.T_ref, -a.beta_P) : 1.0;
  a.beta_P_f = (float)a.beta_P;
  a.T_ref_f = (float)a.T_ref;
  a.tref_mbP_f = (float)a.tref_mbP;
  a.rkJ0 = s->d_rkJ0;
  a.gs_w = s->d_gs;
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
  a.float_quartic = s->params.float_quartic;
  a.k_dcr_f = (float)a.k_dcr;
  a.k_alpha_f = (float)a.k_alpha;
  a.k_g_f = (float)a.k_g;
  a.a_rad_4pi_f = (float)(s->params.a_rad / (4.0 * kPi));
  a.status = s->d_status;
  a.bad_cell = s->d_bad;
  const unsigned blocks = (unsigned)((s->n_cells + CPB - 1) / CPB);
  if constexpr (STAGED) {
    const int cap = stage_cap(s->max_block_slots);
    if (a.float_quartic)
      step_kernel_staged<M, MOVING, QM_FLOAT>
          <<<blocks, NT, stage_bytes(cap, MOVING), s->stream>>>(a, cap);
    else
      step_kernel_staged<M, MOVING, QM_REFINE>
          <<<blocks, NT, stage_bytes(cap, MOVING), s->stream>>>(a, cap);
  } else {
    step_kernel<R, M, MOVING><<<blocks, NT, 0, s->stream>>>(a);
  }
  s->launches++;
  return cudaGetLastError();
}

template <typename R, bool MOVING, bool FULL>
cudaError_t dispatch_pairs(rt_state *s, double dt, const StepIO &io) {
  const int ppt = (s->n_angles / 2 + KT - 1) / KT;
  switch (ppt) {
    case 1: return launch_t<R, PairMap<R, 1, FULL>, MOVING, false>(s, dt, io);
    case 2: return launch_t<R, PairMap<R, 2, FULL>, MOVING, false>(s, dt, io);
    case 3: return launch_t<R, PairMap<R, 3, FULL>, MOVING, false>(s, dt, io);
    case 4: return launch_t<R, PairMap<R, 4, FULL>, MOVING, false>(s, dt, io);
    case 5: return launch_t<R, PairMap<R, 5, FULL>, MOVING, false>(s, dt, io);
    case 6: return launch_t<R, PairMap<R, 6, FULL>, MOVING, false>(s, dt, io);
    case 7: return launch_t<R, PairMap<R, 7, FULL>, MOVING, false>(s, dt, io);
    case 8: return launch_t<R, PairMap<R, 8, FULL>, MOVING, false>(s, dt, io);
    default: return cudaErrorInvalidValue;
  }
}

// Float rows with A = 16 m (32 <= A <= 128) whose blocks' slots fit the
// shared-memory stage: QuadMap<A / 32, A % 32 != 0>.
template <bool MOVING> cudaError_t dispatch_quads(rt_state *s, double dt, const StepIO &io) {
  switch (s->n_angles / 16) {
    case 2: return launch_t<float, QuadMap<1, false>, MOVING, true>(s, dt, io);
    case 3: return launch_t<float, QuadMap<1, true>, MOVING, true>(s, dt, io);
    case 4: return launch_t<float, QuadMap<2, false>, MOVING, true>(s, dt, io);
    case 5: return launch_t<float, QuadMap<2, true>, MOVING, true>(s, dt, io);
    case 6: return launch_t<float, QuadMap<3, false>, MOVING, true>(s, dt, io);
    case 7: return launch_t<float, QuadMap<3, true>, MOVING, true>(s, dt, io);
    case 8: return launch_t<float, QuadMap<4, false>, MOVING, true>(s, dt, io);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R> cudaError_t dispatch(rt_state *s, double dt, const StepIO &io) {
  const int A = s->n_angles;
  if (sizeof(R) == 4 && s->quad_end > 0)  // rows in the quad layout
    return s->moving ? dispatch_quads<true>(s, dt, io) : dispatch_quads<false>(s, dt, io);
  const bool full = (A / 2) % KT == 0;
  if (s->moving)
    return full ? dispatch_pairs<R, true, true>(s, dt, io) : dispatch_pairs<R, true, false>(s, dt, io);
  return full ? dispatch_pairs<R, false, true>(s, dt, io)
              : dispatch_pairs<R, false, false>(s, dt, io);
}

// U[k][p] = the double flux coefficient of pair p through directed face k,
// exactly the expression slot_dot evaluates (cbar A ((n_x n_fx + n_y n_fy) +
// n_z n_fz), rounded in that order): the mesh is fixed for a state's
// lifetime, so the FP64 face loop reads it instead of recomputing it.
__global__ void uface_kernel(const SlotD *__restrict__ slot, const double *__restrict__ dir,
                             int64_t nnz, int H, double *__restrict__ U) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnz * H) return;
  const int64_t k = i / H;
  const int p = (int)(i % H);
  U[i] = slot_dot(dir[4 * p], dir[4 * p + 1], dir[4 * p + 2], load_slot<double>(slot + k));
}

}  // namespace

cudaError_t build_uface(rt_state *s) {
  const int H = s->n_angles / 2;
  const size_t n = (size_t)s->nnz * H;
  if (!s->d_uface) {
    cudaError_t e = cudaMalloc(&s->d_uface, n * sizeof(double));
    if (e != cudaSuccess) return e;
    s->device_bytes += n * sizeof(double);
  }
  const unsigned blocks = (unsigned)((n + 255) / 256);
  uface_kernel<<<blocks, 256, 0, s->stream>>>(reinterpret_cast<const SlotD *>(s->d_slot),
                                              reinterpret_cast<const double *>(s->d_dir), s->nnz, H,
                                              s->d_uface);
  s->launches++;
  return cudaGetLastError();
}

cudaError_t launch_step_io(rt_state *s, double dt, const StepIO &io) {
  return (s->precision == RT_FP32) ? dispatch<float>(s, dt, io) : dispatch<double>(s, dt, io);
}

cudaError_t launch_step(rt_state *s, double dt) {
  cudaError_t e;
  if (s->integrator == RT_VAN_LEER) {
    e = launch_step_vl(s, dt);
  } else if (s->n_groups > 1) {
    // frequency groups: the transport of all groups' intensities and the
    // coupled source step (one fused launch where the layout allows it)
    e = launch_group_step(s, dt, s->d_I[s->cur], s->d_I[s->cur ^ 1]);
  } else {
    const StepIO io{s->d_I[s->cur], s->d_I[s->cur ^ 1], false, true};
    e = launch_step_io(s, dt, io);
  }
  if (e == cudaSuccess) s->cur ^= 1;
  return e;
}

}  // namespace rt
