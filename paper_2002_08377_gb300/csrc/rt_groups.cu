// Implicit source step of frequency groups (Sec. 2.3: groups that share the
// angles and couple only through the gas temperature T^{n+1}), in place on
// the transported rows I*.  Group j owns the angles whose pair index lies in
// [j H, (j+1) H) (H = half the base angle set); its weights are W_j w_a.
//
// Blocks of 32 cells, each warp taking 4 cells in turn with its lanes over
// the row positions of one cell:
//   0  one lane per cell: v / c and every group's x / Gamma = dt cbar
//      (rho kJ_j + rho ks_j);
//   1  per cell and group, the comoving sums of Eq. (Jcom) over the group's
//      angles, S_I,j = sum w~ Gamma^4 I* / (1 + x Gamma), S_G,j and
//      S_1,j = sum w~ / (1 + x Gamma), with w~ = W_j w_a / Gamma^2
//      unnormalised (the normalisation cancels within each group);
//   2  one lane per cell in double: with D_j = S_1,j + dt cbar rho kJ_j S_G,j
//      the temperature equation summed over the groups (Eq. com rad thermal
//      disc), alpha = dt c a sum_j W_j rho kP_j S_1,j / D_j and
//      g = e_int + dt c 4 pi sum_j W_j rho kJ_j S_I,j / D_j, its quartic
//      root, and per group J~_j and q_j = dt cbar rho (kP_j B + ks_j J~_j);
//   3  per cell, the new intensities (Eq. com radiative source disc per
//      group) and the radiation change sum w (I* - I'), sum w n (I* - I');
//   4  one lane per cell in double: the gas exchange (Eqs. gas1, gas2) or the
//      tally of a boundary / emitter cell, and the frame velocity and
//      internal energy of the next step.
// First order in v/c; the grey step handles the boost, the geometric
// conservation law and temperature-dependent opacities.
#include <cuda_runtime.h>

#include "rt_internal.cuh"
#include "rt_step_common.cuh"
#include "rt_step_tile.cuh"

namespace rt {
namespace {

using step::quartic_root;
using step::rcp;

constexpr int kWarps = 8;
constexpr int kCellsPerWarp = 4;
constexpr int kCells = kWarps * kCellsPerWarp;
constexpr int kThreads = 32 * kWarps;
constexpr int kMaxGroups = 8;

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R> struct GroupArgs {
  int64_t n;
  int A, H, Hb, G, quad_end;  // A: all groups' angles, H = A / 2, Hb: H per group
  const GasStatic *gs;
  GasDyn *gd;
  const double *kapg;  // [N][G][3] rho kappa_P, rho kappa_J, rho kappa_s
  const uint8_t *kind;
  const double2 *aux;
  const int32_t *bc_row;
  const R *I0;
  const R *dir;  // [A][4] internal angle order
  const R *wt2;  // [A/2][2]
  R *I;          // [N][A] I* in, I^{n+1} out
  R *cellv;      // [N][4]
  double *ext;   // [N][4]
  double W[kMaxGroups];
  double dt, cbar, a_rad, k_dcr, k_alpha, k_g, k_fe, k_fm;
  R dt_cbar_r, inv_c_r;
  int newton_max_iter;
  int float_quartic;  // float states: 1 solves the temperature equation in float
  unsigned *status;
  unsigned long long *bad_cell;
  // float states (tile kernel): float copies of the group opacities and of
  // the coefficients, W_j dt c a and W_j dt c 4 pi per group
  const float *kapgf;  // [N][G][4]
  float k_dcr_f, a_rad_4pi_f, Wk_alpha_f[kMaxGroups], Wk_g_f[kMaxGroups];
};

template <typename R, int NT> struct Lane {
  R nx[NT], ny[NT], nz[NT], w[NT];
  int q[NT], g[NT];
};

template <typename R, int NT>
__device__ __forceinline__ Lane<R, NT> lane_angles(const GroupArgs<R> &a, int lane) {
  Lane<R, NT> L;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int q = lane + 32 * t;
    L.q[t] = q;
    L.g[t] = -1;
    L.nx[t] = L.ny[t] = L.nz[t] = L.w[t] = R(0);
    if (q < a.A) {
      const int an = angle_of_position(q, a.H, a.quad_end);
      const int p = an < a.H ? an : an - a.H;
      L.g[t] = p / a.Hb;
      L.nx[t] = a.dir[4 * an];
      L.ny[t] = a.dir[4 * an + 1];
      L.nz[t] = a.dir[4 * an + 2];
      L.w[t] = a.wt2[2 * p + (an >= a.H ? 1 : 0)];
    }
  }
  return L;
}

template <typename R> struct CellQ {
  R x[kMaxGroups], q[kMaxGroups];  // per group x / Gamma and q (interior), or Y and Y I_src
  R f;                             // boundary: min(dt / tau, 1)
};

template <typename C> __device__ __forceinline__ C chain_tol();
template <> __device__ __forceinline__ float chain_tol<float>() { return 1e-7f; }
template <> __device__ __forceinline__ double chain_tol<double>() { return 1e-15; }

// Phase 2 of one interior cell in the compute type C: with D_j = S_1,j +
// dt cbar rho kJ_j S_G,j, the group-weighted quartic alpha T^4 + rho c_v T = g
// and every group's q_j.  Returns the status bits, or -1 when a result is
// not finite (the caller then repeats it in double).
template <typename C, typename R>
__device__ int group_chain(const GroupArgs<R> &a, int64_t cl, const double (*sm)[3], double eint,
                           double rcv, C *q) {
  const int G = a.G;
  C alpha = 0, gq = C(eint), rU[kMaxGroups];
  for (int j = 0; j < G; ++j) {
    const double *k = a.kapg + ((size_t)cl * G + j) * 3;
    rU[j] = C(1) / fma(C(a.k_dcr * k[1]), C(sm[j][1]), C(sm[j][2]));
    alpha += C(a.W[j] * a.k_alpha * k[0]) * C(sm[j][2]) * rU[j];
    gq += C(a.W[j] * a.k_g * k[1]) * C(sm[j][0]) * rU[j];
  }
  if (!(gq >= C(0)) || !(alpha >= C(0))) return sizeof(C) == 4 ? -1 : (int)ST_NONFINITE;
  C T;
  const int nc = quartic_root(alpha, C(rcv), gq, C(eint / rcv), chain_tol<C>(), a.newton_max_iter, &T);
  const C B = C(a.a_rad * (1.0 / (4.0 * kPi))) * (T * T) * (T * T);
  for (int j = 0; j < G; ++j) {
    const double *k = a.kapg + ((size_t)cl * G + j) * 3;
    const C dP = C(a.k_dcr * k[0]), dS = C(a.k_dcr * k[2]);
    const C J = fma(dP * B, C(sm[j][1]), C(sm[j][0])) * rU[j];
    q[j] = fma(dP, B, dS * J);
    if (sizeof(C) == 4 && !isfinite(q[j])) return -1;
  }
  return nc ? (int)ST_NONCONV : 0;
}

// The temperature equation of one interior cell in float from float inputs
// (tile kernel, float states): per group rho kP_j, rho kJ_j, rho ks_j in kf
// and the sums S_I,j, S_G,j, S_1,j.  group_coeffs_f forms alpha, g and the
// 1 / D_j (false when they are negative or not finite); group_q_f forms every
// group's q_j from a root T (false when one is not finite); group_chain_f
// solves the quartic in float between the two, returning the status bits, or
// -1 when a result is not finite (the caller then takes group_chain<double>).
constexpr int kTileGroups = 4;
struct GroupQuarticF {
  float alpha, gq, rU[kTileGroups];
};
__device__ __forceinline__ bool group_coeffs_f(const GroupArgs<float> &a,
                                               const float4 (&kf)[kTileGroups],
                                               const float (&SI)[kTileGroups],
                                               const float (&SG)[kTileGroups],
                                               const float (&S1)[kTileGroups], float eint,
                                               GroupQuarticF &k) {
  k.alpha = 0.0f;
  k.gq = eint;
#pragma unroll
  for (int j = 0; j < kTileGroups; ++j) {
    k.rU[j] = 0.0f;
    if (j < a.G) {
      k.rU[j] = rcp(fmaf(a.k_dcr_f * kf[j].y, SG[j], S1[j]));
      k.alpha = fmaf(a.Wk_alpha_f[j] * kf[j].x * S1[j], k.rU[j], k.alpha);
      k.gq = fmaf(a.Wk_g_f[j] * kf[j].y * SI[j], k.rU[j], k.gq);
    }
  }
  return k.gq >= 0.0f && k.alpha >= 0.0f && isfinite(k.alpha) && isfinite(k.gq);
}
__device__ __forceinline__ bool group_q_f(const GroupArgs<float> &a,
                                          const float4 (&kf)[kTileGroups],
                                          const float (&SI)[kTileGroups],
                                          const float (&SG)[kTileGroups], const GroupQuarticF &k,
                                          float T, float (&q)[kTileGroups]) {
  const float B = a.a_rad_4pi_f * (T * T) * (T * T);
  bool ok = true;
#pragma unroll
  for (int j = 0; j < kTileGroups; ++j) {
    q[j] = 0.0f;
    if (j < a.G) {
      const float dP = a.k_dcr_f * kf[j].x, dS = a.k_dcr_f * kf[j].z;
      const float J = fmaf(dP * B, SG[j], SI[j]) * k.rU[j];
      q[j] = fmaf(dP, B, dS * J);
      ok = ok && isfinite(q[j]);
    }
  }
  return ok;
}
__device__ __forceinline__ int group_chain_f(const GroupArgs<float> &a, const float4 (&kf)[kTileGroups],
                                             const float (&SI)[kTileGroups],
                                             const float (&SG)[kTileGroups],
                                             const float (&S1)[kTileGroups], float eint, float rcv,
                                             float (&q)[kTileGroups]) {
  GroupQuarticF k;
  if (!group_coeffs_f(a, kf, SI, SG, S1, eint, k)) return -1;
  float T;
  const int nc = quartic_root(k.alpha, rcv, k.gq, eint * rcp(rcv), 1e-7f, a.newton_max_iter, &T);
  if (!group_q_f(a, kf, SI, SG, k, T, q)) return -1;
  return nc ? (int)ST_NONCONV : 0;
}
// The float opacities of a cell's groups (zero past G).
__device__ __forceinline__ void load_kf(const GroupArgs<float> &a, int64_t c,
                                        float4 (&kf)[kTileGroups]) {
#pragma unroll
  for (int g = 0; g < kTileGroups; ++g)
    kf[g] = g < a.G ? reinterpret_cast<const float4 *>(a.kapgf)[(size_t)c * a.G + g]
                    : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

template <typename R, int NT>
__global__ void __launch_bounds__(kThreads) group_source_kernel(const GroupArgs<R> a) {
  __shared__ R bx_s[kCells], by_s[kCells], bz_s[kCells];
  __shared__ int kind_s[kCells];
  __shared__ double sums[kCells][kMaxGroups][3];  // S_I, S_G, S_1 per group
  __shared__ CellQ<R> cq[kCells];
  __shared__ double dEF[kCells][4];
  __shared__ unsigned bad_s[kCells];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t c0 = (int64_t)blockIdx.x * kCells;
  const int64_t cl = c0 + lane;
  const bool lane_cell = warp == 0 && cl < a.n;
  const int G = a.G;

  // ---------------- phase 0
  if (lane_cell) {
    const GasStatic gs = a.gs[cl];
    const GasDyn d = a.gd[cl];
    const int kind = a.kind[cl];
    kind_s[lane] = kind;
    bx_s[lane] = R(d.mx * gs.inv_rho) * a.inv_c_r;
    by_s[lane] = R(d.my * gs.inv_rho) * a.inv_c_r;
    bz_s[lane] = R(d.mz * gs.inv_rho) * a.inv_c_r;
    bad_s[lane] = 0;
    CellQ<R> &Q = cq[lane];
    for (int j = 0; j < G; ++j) {
      const double *k = a.kapg + ((size_t)cl * G + j) * 3;
      Q.x[j] = a.dt_cbar_r * R(k[1] + k[2]);
      Q.q[j] = R(0);
    }
    Q.f = R(0);
    if (kind == RT_CELL_BOUNDARY) {
      const double2 ax = a.aux[cl];
      Q.f = R((ax.x <= a.dt) ? 1.0 : a.dt / ax.x);
    } else if (kind == RT_CELL_EMITTER) {
      const double2 ax = a.aux[cl];
      const R Y = R(a.dt * a.cbar * ax.x);
      for (int j = 0; j < G; ++j) {
        Q.x[j] = Y;
        Q.q[j] = Y * R(ax.y);
      }
    }
  }
  __syncthreads();

  const Lane<R, NT> L = lane_angles<R, NT>(a, lane);
  R is[kCellsPerWarp][NT];
#pragma unroll
  for (int i = 0; i < kCellsPerWarp; ++i) {
    const int64_t c = c0 + warp * kCellsPerWarp + i;
#pragma unroll
    for (int t = 0; t < NT; ++t)
      is[i][t] = c < a.n && L.q[t] < a.A ? a.I[(size_t)c * a.A + L.q[t]] : R(0);
  }

  // ---------------- phase 1: per-group comoving sums of interior cells
#pragma unroll
  for (int i = 0; i < kCellsPerWarp; ++i) {
    const int lc = warp * kCellsPerWarp + i;
    if (c0 + lc >= a.n || kind_s[lc] != RT_CELL_INTERIOR) continue;
    const R bx = bx_s[lc], by = by_s[lc], bz = bz_s[lc];
    R sI[NT], sG[NT], s1[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      sI[t] = sG[t] = s1[t] = R(0);
      if (L.q[t] < a.A) {
        const R Gm = R(1) - fma(bx, L.nx[t], fma(by, L.ny[t], bz * L.nz[t]));
        const R G2 = Gm * Gm;
        const R tw = L.w[t] * rcp(G2 * fma(cq[lc].x[L.g[t]], Gm, R(1)));  // w~ / (1 + x Gamma)
        s1[t] = tw;
        sI[t] = tw * G2 * G2 * is[i][t];
        sG[t] = tw * Gm;
      }
    }
    for (int j = 0; j < G; ++j) {
      R pI = 0, pG = 0, p1 = 0;
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (L.g[t] == j) {
          pI += sI[t];
          pG += sG[t];
          p1 += s1[t];
        }
      // reduced in the state precision (a double reduction costs FP64 adds)
      const R SI = warp_sum(pI), SG = warp_sum(pG), S1 = warp_sum(p1);
      if (lane == 0) {
        sums[lc][j][0] = SI;
        sums[lc][j][1] = SG;
        sums[lc][j][2] = S1;
      }
    }
  }
  __syncthreads();

  // ---------------- phase 2: the temperature equation over all groups
  if (lane_cell && kind_s[lane] == RT_CELL_INTERIOR) {
    const GasStatic gs = a.gs[cl];
    const GasDyn d = a.gd[cl];
    const double eint = d.e - 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * gs.inv_rho;
    unsigned bad = 0;
    bool done = false;
    if (sizeof(R) == 4 && a.float_quartic) {
      // float states with float_quartic: the chain in float, as the grey
      // float step then solves its quartic; repeated in double if a result
      // is not finite
      float q[kMaxGroups];
      const int st = group_chain<float>(a, cl, sums[lane], eint, gs.rcv, q);
      if (st >= 0) {
        for (int j = 0; j < G; ++j) cq[lane].q[j] = q[j];
        bad = st;
        done = true;
      }
    }
    if (!done) {
      double q[kMaxGroups];
      const int st = group_chain<double>(a, cl, sums[lane], eint, gs.rcv, q);
      for (int j = 0; j < G; ++j) cq[lane].q[j] = R(q[j]);
      bad = st < 0 ? ST_NONFINITE : (unsigned)st;
    }
    bad_s[lane] = bad;
  }
  __syncthreads();

  // ---------------- phase 3: new intensities and the radiation change
#pragma unroll
  for (int i = 0; i < kCellsPerWarp; ++i) {
    const int lc = warp * kCellsPerWarp + i;
    const int64_t c = c0 + lc;
    if (c >= a.n) continue;
    const int kind = kind_s[lc];
    const R bx = bx_s[lc], by = by_s[lc], bz = bz_s[lc];
    const R *I0row = kind == RT_CELL_BOUNDARY ? a.I0 + (size_t)a.bc_row[c] * a.A : nullptr;
    R de = 0, dfx = 0, dfy = 0, dfz = 0;
#pragma unroll
    for (int t = 0; t < NT; ++t)
      if (L.q[t] < a.A) {
        const R Is = is[i][t];
        R In, dI;  // dI: the change I* - I' the gas receives (see the tile kernel)
        if (kind == RT_CELL_BOUNDARY) {
          In = fma(-cq[lc].f, Is - I0row[L.q[t]], Is);
          dI = sizeof(R) == 8 ? cq[lc].f * (Is - I0row[L.q[t]]) : Is - In;
        } else {
          // I' = (I* Gamma^3 + q) / (Gamma^3 (1 + x Gamma))
          const R Gm = R(1) - fma(bx, L.nx[t], fma(by, L.ny[t], bz * L.nz[t]));
          const R G3 = Gm * Gm * Gm;
          const int j = L.g[t];
          if constexpr (sizeof(R) == 8) {
            const R xg = cq[lc].x[j] * Gm, r = rcp(G3 * (xg + R(1))), tI = Is * G3;
            In = (tI + cq[lc].q[j]) * r;
            dI = fma(tI, xg, -cq[lc].q[j]) * r;
          } else {
            In = fma(Is, G3, cq[lc].q[j]) * rcp(G3 * fma(cq[lc].x[j], Gm, R(1)));
            dI = Is - In;
          }
        }
        a.I[(size_t)c * a.A + L.q[t]] = In;
        const R dw = L.w[t] * dI;
        de += dw;
        dfx = fma(L.nx[t], dw, dfx);
        dfy = fma(L.ny[t], dw, dfy);
        dfz = fma(L.nz[t], dw, dfz);
      }
    const R sE = warp_sum(de), sx = warp_sum(dfx), sy = warp_sum(dfy), sz = warp_sum(dfz);
    if (lane == 0) {
      dEF[lc][0] = sE;
      dEF[lc][1] = sx;
      dEF[lc][2] = sy;
      dEF[lc][3] = sz;
    }
  }
  __syncthreads();

  // ---------------- phase 4: gas exchange, one lane per cell
  if (lane_cell) {
    const double dE = a.k_fe * dEF[lane][0];
    const double dx = a.k_fm * dEF[lane][1], dy = a.k_fm * dEF[lane][2], dz = a.k_fm * dEF[lane][3];
    unsigned bad = bad_s[lane];
    if (!isfinite(dE)) bad |= ST_NONFINITE;
    if (kind_s[lane] == RT_CELL_INTERIOR) {
      GasDyn d = a.gd[cl];
      d.e += dE;
      d.mx += dx;
      d.my += dy;
      d.mz += dz;
      a.gd[cl] = d;
      const double ir = a.gs[cl].inv_rho;
      const double kin = 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * ir;
      R *cv = a.cellv + 4 * cl;
      cv[0] = R(d.mx * ir);
      cv[1] = R(d.my * ir);
      cv[2] = R(d.mz * ir);
      cv[3] = R(d.e - kin);
    } else {
      double *x = a.ext + 4 * cl;
      x[0] += dE;
      x[1] += dx;
      x[2] += dy;
      x[3] += dz;
    }
    if (bad) {
      atomicOr(a.status, bad);
      atomicMin(a.bad_cell, (unsigned long long)cl);
    }
  }
}

// ------------------------------------------------------------ tile kernel
// The same step for up to kTileGroups groups on the step kernel's tile
// mapping (blocks of 32 cells x 8 threads, a thread owning the pairs of its
// pair / quad map).  The group of pair p is p / Hb, and every sum is kept
// per group (unused groups stay zero).  Float states find the root of the
// temperature equation in float in all 8 lanes of a cell, from float copies
// of the group opacities; by default one lane per cell then refines it by a
// Newton step in double between two block barriers and forms the groups' q_j
// (float_quartic = 1 keeps the float root, with no barrier); where a float
// result is not finite the double chain runs instead.  Double states solve
// it one lane per cell in double between two barriers.  The gas exchange is
// one lane per cell in double after a barrier, as in the grey step.
template <typename R> struct TileShared {
  double s[CPB][kTileGroups][3];  // S_I, S_G, S_1 per group
  R q[CPB][kTileGroups];
  float qT[CPB];                  // float states: the in-lane float root
  unsigned fst[CPB];              // float states: 0 when that root is usable
  R dE[CPB], dF[3][CPB];
  unsigned bad[CPB];
};

// rho kappa_J + rho kappa_s of group g of cell c, in the state precision
__device__ __forceinline__ float group_xs(const GroupArgs<float> &a, int64_t c, int g) {
  const float4 k = reinterpret_cast<const float4 *>(a.kapgf)[(size_t)c * a.G + g];
  return k.y + k.z;
}
__device__ __forceinline__ double group_xs(const GroupArgs<double> &a, int64_t c, int g) {
  const double *k = a.kapg + ((size_t)c * a.G + g) * 3;
  return k[1] + k[2];
}

// The group step's body for the thread's entries.  FUSED (float rows in the
// quad layout, static mesh): the transport runs first in the same block --
// the block's face slots staged in shared memory, I* = I^n - dt/V sum_f u I_up
// formed in registers from t.I_in -- so the transported rows never go
// through memory; a.I then receives I^{n+1}.  Otherwise a.I holds I* and is
// updated in place.
template <typename R, typename M, bool FUSED>
__device__ __forceinline__ void group_tile_body(const GroupArgs<R> &a, const StepArgs<R> &t,
                                                const step::StageView &stage);

template <typename R, typename M>
__global__ void __launch_bounds__(step::NT, sizeof(R) == 4 && M::PPT <= 6 ? 3 : 2)
    group_source_tile(const GroupArgs<R> a) {
  group_tile_body<R, M, false>(a, StepArgs<R>{}, step::StageView{});
}

template <typename M>
__global__ void __launch_bounds__(step::NT, M::PPT <= 6 ? 3 : 2)
    group_step_fused(const GroupArgs<float> a, const StepArgs<float> t, int cap) {
  extern __shared__ __align__(128) unsigned char dyn[];
  const step::StageView v = step::stage_at(dyn, cap, false);
  step::issue_stage<false, false>(t, blockIdx.x, v);
  group_tile_body<float, M, true>(a, t, v);
}

template <typename R, typename M, bool FUSED>
__device__ __forceinline__ void group_tile_body(const GroupArgs<R> &a, const StepArgs<R> &t,
                                                const step::StageView &stage) {
  using V = step::pair_t<R>;
  using step::mk;
  using step::padd;
  using step::pfma;
  using step::pmul;
  using step::psub;
  constexpr int PPT = M::PPT;
  constexpr int NG = kTileGroups;
  __shared__ TileShared<R> sh;
  const int lc = threadIdx.x / step::KT, sub = threadIdx.x % step::KT;
  const int64_t cell = (int64_t)blockIdx.x * CPB + lc;
  const bool live = cell < a.n;
  const int64_t c = live ? cell : a.n - 1;  // dead lanes shadow the last cell
  const int np = M::count(a.H, sub);
  R Ia[PPT], Ib[PPT], nx[PPT], ny[PPT], nz[PPT];
  int gp[PPT];
  M::load((FUSED ? t.I_in : a.I) + (size_t)c * a.A, sub, Ia, Ib, np);
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int p = (M::FULL || j < np) ? M::pair(j, sub) : 0;
    step::load_dir(a.dir, p, nx[j], ny[j], nz[j]);
    gp[j] = p / a.Hb;
  }
  if constexpr (FUSED) {
    // I* of the thread's entries: the step kernel's face loop over the
    // block's staged slots, in the cell's face order
    R acca[PPT], accb[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) acca[j] = accb[j] = R(0);
    const int64_t kb = t.ptr[(int64_t)blockIdx.x * CPB];
    const int k0 = (int)(t.ptr[c] - kb), k1 = (int)(t.ptr[c + 1] - kb);
    step::cp_async_wait_all();
    __syncthreads();  // the block's stage has landed
    step::face_sum<R, M, false, true, step::TRANSPORT_FORWARD>(
        reinterpret_cast<const typename SlotOf<R>::type *>(stage.slot), stage.nbr, t.wface,
        t.uface, t.half, k0, k1, t.I_in, t.row, sub, nx, ny, nz, Ia, Ib, acca, accb, np);
    const R dtv = t.dt_r * t.inv_vol[c];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      Ia[j] = fma(-dtv, acca[j], Ia[j]);
      Ib[j] = fma(-dtv, accb[j], Ib[j]);
    }
  }
  const int kind = a.kind[c];
  const R vxc = a.cellv[4 * c] * a.inv_c_r, vyc = a.cellv[4 * c + 1] * a.inv_c_r,
          vzc = a.cellv[4 * c + 2] * a.inv_c_r;
  R xs[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) xs[g] = g < a.G ? a.dt_cbar_r * R(group_xs(a, c, g)) : R(0);
  const V *W2 = reinterpret_cast<const V *>(a.wt2);
  const V one = mk(R(1), R(1));

  // ---------------- phase A: per-group comoving sums (interior cells)
  V sIv[NG], sGv[NG], s1v[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) sIv[g] = sGv[g] = s1v[g] = mk(R(0), R(0));
  if (kind == RT_CELL_INTERIOR) {
#pragma unroll
    for (int j = 0; j < PPT; ++j)
      if (M::FULL || j < np) {
        R xg = xs[0];
#pragma unroll
        for (int g = 1; g < NG; ++g) xg = gp[j] == g ? xs[g] : xg;
        const R bn = fma(vxc, nx[j], fma(vyc, ny[j], vzc * nz[j]));
        const V Gv = mk(R(1) - bn, R(1) + bn);
        const V G2 = pmul(Gv, Gv);
        const V t = pmul(W2[M::pair(j, sub)], step::prcp<R>(pmul(G2, pfma(mk(xg, xg), Gv, one))));
        const V tI = pmul(pmul(t, pmul(G2, G2)), mk(Ia[j], Ib[j]));
        const V tG = pmul(t, Gv);
#pragma unroll
        for (int g = 0; g < NG; ++g)
          if (gp[j] == g) {
            s1v[g] = padd(s1v[g], t);
            sIv[g] = padd(sIv[g], tI);
            sGv[g] = padd(sGv[g], tG);
          }
      }
  }
  R sI[NG], sG[NG], s1[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    sI[g] = step::cell_sum(sIv[g].x + sIv[g].y);
    sG[g] = step::cell_sum(sGv[g].x + sGv[g].y);
    s1[g] = step::cell_sum(s1v[g].x + s1v[g].y);
  }


  // ---------------- phase B: the temperature equation over all groups
  R q[NG];
  unsigned bad = 0;
#pragma unroll
  for (int g = 0; g < NG; ++g) q[g] = R(0);
  bool lane_solve = false;  // float states with float_quartic: in float, in every lane
  if constexpr (sizeof(R) == 4) lane_solve = a.float_quartic != 0;
  if (lane_solve) {
    if constexpr (sizeof(R) == 4) if (kind == RT_CELL_INTERIOR) {
      float4 kf[NG];
      load_kf(a, c, kf);
      const int st = group_chain_f(a, kf, sI, sG, s1, a.cellv[4 * c + 3], a.gs[c].frcv, q);
      if (st >= 0) {
        bad = st;
      } else {
        double sm[kMaxGroups][3], qd[kMaxGroups];
        for (int g = 0; g < a.G && g < NG; ++g) {
          sm[g][0] = sI[g];
          sm[g][1] = sG[g];
          sm[g][2] = s1[g];
        }
        const GasDyn d = a.gd[c];
        const GasStatic gs = a.gs[c];
        const double eint = d.e - 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * gs.inv_rho;
        bad = group_chain<double>(a, c, sm, eint, gs.rcv, qd);
#pragma unroll
        for (int g = 0; g < NG; ++g) q[g] = g < a.G ? R(qd[g]) : R(0);
      }
    }
  } else {
    // float states (default): every lane finds the float root of the
    // temperature equation from the float sums (no barrier); one lane per
    // cell then refines it by a Newton step in double (the FP64 temperature
    // solve) and forms the groups' q_j in float from it, or, where the float
    // solve failed, runs the whole double chain.  Double states: the double
    // chain, one lane per cell.
    float Tf = 0.0f;
    unsigned fst = 1;
    if constexpr (sizeof(R) == 4) if (kind == RT_CELL_INTERIOR) {
      float4 kf[NG];
      load_kf(a, c, kf);
      GroupQuarticF k;
      const float eint = a.cellv[4 * c + 3], rcv = a.gs[c].frcv;
      if (group_coeffs_f(a, kf, sI, sG, s1, eint, k) &&
          !quartic_root(k.alpha, rcv, k.gq, eint * rcp(rcv), 1e-7f, a.newton_max_iter, &Tf) &&
          isfinite(Tf))
        fst = 0;
    }
    if (sub == 0) {
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        sh.s[lc][g][0] = sI[g];
        sh.s[lc][g][1] = sG[g];
        sh.s[lc][g][2] = s1[g];
      }
      sh.qT[lc] = Tf;
      sh.fst[lc] = fst;
    }
    __syncthreads();
    if (threadIdx.x < CPB) {
      const int lp = threadIdx.x;
      const int64_t cl = (int64_t)blockIdx.x * CPB + lp;
      unsigned bl = 0;
      bool done = false;
      if constexpr (sizeof(R) == 4)
        if (cl < a.n && a.kind[cl] == RT_CELL_INTERIOR && sh.fst[lp] == 0) {
          float4 kf[NG];
          load_kf(a, cl, kf);
          float SI[NG], SG[NG], S1[NG];
#pragma unroll
          for (int g = 0; g < NG; ++g) {
            SI[g] = (float)sh.s[lp][g][0];
            SG[g] = (float)sh.s[lp][g][1];
            S1[g] = (float)sh.s[lp][g][2];
          }
          GroupQuarticF k;  // the in-lane coefficients, formed again from the same floats
          group_coeffs_f(a, kf, SI, SG, S1, a.cellv[4 * cl + 3], k);
          const double T =
              step::refine_root(k.alpha, 0.0f, 0.0, a.gs[cl].rcv, k.gq, sh.qT[lp]);
          float qf[NG];
          if (group_q_f(a, kf, SI, SG, k, (float)T, qf)) {
#pragma unroll
            for (int g = 0; g < NG; ++g)
              if (g < a.G) sh.q[lp][g] = qf[g];
            done = true;
          }
        }
      if (!done && cl < a.n && a.kind[cl] == RT_CELL_INTERIOR) {
        const GasDyn d = a.gd[cl];
        const GasStatic gs = a.gs[cl];
        const double eint = d.e - 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * gs.inv_rho;
        double qd[kMaxGroups];
        bl = group_chain<double>(a, cl, sh.s[lp], eint, gs.rcv, qd);
        for (int g = 0; g < a.G && g < NG; ++g) sh.q[lp][g] = R(qd[g]);
      }
      sh.bad[lp] = bl;
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < NG; ++g) q[g] = g < a.G ? sh.q[lc][g] : R(0);
    bad = sh.bad[lc];
  }

  // ---------------- phase C: new intensities and the radiation change
  // The change I* - I' the gas receives: float states take the difference
  // of the stored intensities (exact energy bookkeeping in float), double
  // states the source term itself (rounding relative to the change), as the
  // grey step kernel does.
  R na[PPT], nb[PPT];
  constexpr int ND = sizeof(R) == 8 ? PPT : 1;
  R da[ND], db[ND];
  if (kind == RT_CELL_BOUNDARY) {
    const double2 ax = a.aux[c];
    const R f = R((ax.x <= a.dt) ? 1.0 : a.dt / ax.x);
    R tx[PPT], ty[PPT];
    M::load(a.I0 + (size_t)a.bc_row[c] * a.A, sub, tx, ty, np);
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
    // I' = (I* Gamma^3 + q) / (Gamma^3 (1 + x Gamma)); emitters: x -> dt cbar
    // (rho kappa)_src and q -> that rate times I_src in every group
    const bool em = kind == RT_CELL_EMITTER;
    R xe = R(0), qe = R(0);
    if (em) {
      const double2 ax = a.aux[c];
      xe = R(a.dt * a.cbar * ax.x);
      qe = xe * R(ax.y);
    }
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      R xg = xs[0], qg = q[0];
#pragma unroll
      for (int g = 1; g < NG; ++g) {
        xg = gp[j] == g ? xs[g] : xg;
        qg = gp[j] == g ? q[g] : qg;
      }
      if (em) {
        xg = xe;
        qg = qe;
      }
      const R bn = fma(vxc, nx[j], fma(vyc, ny[j], vzc * nz[j]));
      const V Gv = mk(R(1) - bn, R(1) + bn);
      const V G3 = pmul(pmul(Gv, Gv), Gv);
      if constexpr (sizeof(R) == 8) {
        const V XG = pmul(mk(xg, xg), Gv);
        const V r = step::prcp<R>(pmul(G3, padd(XG, one)));
        const V t = pmul(mk(Ia[j], Ib[j]), G3);
        const V n = pmul(padd(t, mk(qg, qg)), r);
        const V d = pmul(pfma(t, XG, mk(-qg, -qg)), r);
        na[j] = n.x;
        nb[j] = n.y;
        da[j] = d.x;
        db[j] = d.y;
      } else {
        const V n = pmul(pfma(mk(Ia[j], Ib[j]), G3, mk(qg, qg)),
                         step::prcp<R>(pmul(G3, pfma(mk(xg, xg), Gv, one))));
        na[j] = n.x;
        nb[j] = n.y;
      }
    }
  }
  if (live) M::store(a.I + (size_t)c * a.A, sub, na, nb, np);
  V dev = mk(R(0), R(0));
  R dfx = 0, dfy = 0, dfz = 0;
#pragma unroll
  for (int j = 0; j < PPT; ++j)
    if (M::FULL || j < np) {
      V d;
      if constexpr (sizeof(R) == 8)
        d = pmul(W2[M::pair(j, sub)], mk(da[j], db[j]));
      else
        d = pmul(W2[M::pair(j, sub)], psub(mk(Ia[j], Ib[j]), mk(na[j], nb[j])));
      dev = padd(dev, d);
      const R df = d.x - d.y;  // the antipode has direction -n
      dfx = fma(nx[j], df, dfx);
      dfy = fma(ny[j], df, dfy);
      dfz = fma(nz[j], df, dfz);
    }
  R de = step::cell_sum(dev.x + dev.y);
  dfx = step::cell_sum(dfx);
  dfy = step::cell_sum(dfy);
  dfz = step::cell_sum(dfz);
  const unsigned nonfinite = step::cell_or(isfinite(de) ? 0u : (unsigned)ST_NONFINITE);
  if (sub == 0) {
    sh.dE[lc] = de;
    sh.dF[0][lc] = dfx;
    sh.dF[1][lc] = dfy;
    sh.dF[2][lc] = dfz;
    sh.bad[lc] = bad | nonfinite;
  }
  __syncthreads();

  // ---------------- phase D: gas exchange (Eqs. gas1, gas2), one lane per cell
  if (threadIdx.x < CPB) {
    const int lp = threadIdx.x;
    const int64_t cl = (int64_t)blockIdx.x * CPB + lp;
    if (cl < a.n) {
      const double dE = a.k_fe * (double)sh.dE[lp];
      const double dx = a.k_fm * (double)sh.dF[0][lp], dy = a.k_fm * (double)sh.dF[1][lp],
                   dz = a.k_fm * (double)sh.dF[2][lp];
      if (a.kind[cl] == RT_CELL_INTERIOR) {
        GasDyn d = a.gd[cl];
        d.e += dE;
        d.mx += dx;
        d.my += dy;
        d.mz += dz;
        a.gd[cl] = d;
        const double ir = a.gs[cl].inv_rho;
        const double kin = 0.5 * (d.mx * d.mx + d.my * d.my + d.mz * d.mz) * ir;
        step::store4(a.cellv + 4 * cl, R(d.mx * ir), R(d.my * ir), R(d.mz * ir), R(d.e - kin));
      } else {
        double *x = a.ext + 4 * cl;
        x[0] += dE;
        x[1] += dx;
        x[2] += dy;
        x[3] += dz;
      }
      const unsigned b = sh.bad[lp];
      if (b) {
        atomicOr(a.status, b);
        atomicMin(a.bad_cell, (unsigned long long)cl);
      }
    }
  }
}

template <typename R, typename M> void launch_tile(const GroupArgs<R> &a, cudaStream_t st) {
  const unsigned g = (unsigned)((a.n + CPB - 1) / CPB);
  group_source_tile<R, M><<<g, step::NT, 0, st>>>(a);
}

template <typename R, bool FULL> void tile_pairs(const GroupArgs<R> &a, cudaStream_t st) {
  switch ((a.H + step::KT - 1) / step::KT) {
    case 1: launch_tile<R, step::PairMap<R, 1, FULL>>(a, st); break;
    case 2: launch_tile<R, step::PairMap<R, 2, FULL>>(a, st); break;
    case 3: launch_tile<R, step::PairMap<R, 3, FULL>>(a, st); break;
    case 4: launch_tile<R, step::PairMap<R, 4, FULL>>(a, st); break;
    case 5: launch_tile<R, step::PairMap<R, 5, FULL>>(a, st); break;
    case 6: launch_tile<R, step::PairMap<R, 6, FULL>>(a, st); break;
    case 7: launch_tile<R, step::PairMap<R, 7, FULL>>(a, st); break;
    default: launch_tile<R, step::PairMap<R, 8, FULL>>(a, st); break;
  }
}

// the map of the state's row layout (quads for float rows in the quad layout)
template <typename R> void tile_dispatch(const GroupArgs<R> &a, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {
    if (a.quad_end > 0) {
      switch (a.A / 16) {
        case 2: launch_tile<float, step::QuadMap<1, false>>(a, st); return;
        case 3: launch_tile<float, step::QuadMap<1, true>>(a, st); return;
        case 4: launch_tile<float, step::QuadMap<2, false>>(a, st); return;
        case 5: launch_tile<float, step::QuadMap<2, true>>(a, st); return;
        case 6: launch_tile<float, step::QuadMap<3, false>>(a, st); return;
        case 7: launch_tile<float, step::QuadMap<3, true>>(a, st); return;
        default: launch_tile<float, step::QuadMap<4, false>>(a, st); return;
      }
    }
  }
  if (a.H % step::KT == 0)
    tile_pairs<R, true>(a, st);
  else
    tile_pairs<R, false>(a, st);
}

template <typename R> GroupArgs<R> group_args(rt_state *s, double dt, void *Is) {
  GroupArgs<R> a{};
  a.n = s->n_cells;
  a.A = s->n_angles;
  a.H = a.A / 2;
  a.G = s->n_groups;
  a.Hb = a.H / a.G;
  a.quad_end = s->quad_end;
  a.gs = s->d_gs;
  a.gd = s->d_gd;
  a.kapg = s->d_kapg;
  a.kind = s->d_kind;
  a.aux = s->d_aux;
  a.bc_row = s->d_bc_row;
  a.I0 = reinterpret_cast<const R *>(s->d_I0);
  a.dir = reinterpret_cast<const R *>(s->d_dir);
  a.wt2 = reinterpret_cast<const R *>(s->d_wt);
  a.I = reinterpret_cast<R *>(Is);
  a.cellv = reinterpret_cast<R *>(s->d_cellv);
  a.ext = s->d_ext;
  for (int j = 0; j < a.G && j < kMaxGroups; ++j) a.W[j] = s->group_w[j];
  a.dt = dt;
  a.cbar = s->params.cbar;
  a.a_rad = s->params.a_rad;
  a.k_dcr = dt * s->params.cbar;
  a.k_alpha = dt * s->params.c * s->params.a_rad;
  a.k_g = dt * s->params.c * 4.0 * kPi;
  a.k_fe = s->params.c / s->params.cbar * 4.0 * kPi;
  a.k_fm = 4.0 * kPi / s->params.cbar;
  a.dt_cbar_r = R(dt * s->params.cbar);
  a.inv_c_r = R(1.0 / s->params.c);
  a.newton_max_iter = s->params.newton_max_iter;
  a.float_quartic = s->params.float_quartic;
  a.status = s->d_status;
  a.bad_cell = s->d_bad;
  a.kapgf = s->d_kapgf;
  a.k_dcr_f = (float)a.k_dcr;
  a.a_rad_4pi_f = (float)(s->params.a_rad / (4.0 * kPi));
  for (int j = 0; j < a.G && j < kMaxGroups; ++j) {
    a.Wk_alpha_f[j] = (float)(a.W[j] * a.k_alpha);
    a.Wk_g_f[j] = (float)(a.W[j] * a.k_g);
  }
  return a;
}

template <typename R> cudaError_t launch(rt_state *s, double dt, void *Is) {
  const GroupArgs<R> a = group_args<R>(s, dt, Is);
  if (a.G <= kTileGroups) {
    tile_dispatch<R>(a, s->stream);
    s->launches++;
    return cudaGetLastError();
  }
  const unsigned g = (unsigned)((a.n + kCells - 1) / kCells);
  switch ((a.A + 31) / 32) {
    case 1: group_source_kernel<R, 1><<<g, kThreads, 0, s->stream>>>(a); break;
    case 2: group_source_kernel<R, 2><<<g, kThreads, 0, s->stream>>>(a); break;
    case 3: group_source_kernel<R, 3><<<g, kThreads, 0, s->stream>>>(a); break;
    default: group_source_kernel<R, 4><<<g, kThreads, 0, s->stream>>>(a); break;
  }
  s->launches++;
  return cudaGetLastError();
}

template <typename M>
cudaError_t launch_fused_q(rt_state *s, double dt, const void *In, void *Out) {
  const GroupArgs<float> a = group_args<float>(s, dt, Out);
  StepArgs<float> t{};
  t.n_cells = s->n_cells;
  t.n_angles = s->n_angles;
  t.half = s->n_angles / 2;
  t.row = s->row_stride;
  t.ptr = s->d_ptr;
  t.nbr = s->d_nbr;
  t.slot = reinterpret_cast<const SlotF *>(s->d_slot);
  t.slot_nb = s->d_slot_nb;
  t.uface = s->d_uface;
  t.inv_vol = reinterpret_cast<const float *>(s->d_inv_vol);
  t.wface = s->d_wface;
  t.dir = reinterpret_cast<const float *>(s->d_dir);
  t.I_in = reinterpret_cast<const float *>(In);
  t.I_out = nullptr;
  t.dt = dt;
  t.dt_r = (float)dt;
  const unsigned g = (unsigned)((s->n_cells + CPB - 1) / CPB);
  const int cap = step::stage_cap(s->max_block_slots);
  group_step_fused<M><<<g, step::NT, step::stage_gas_offset(cap, false), s->stream>>>(a, t, cap);
  s->launches++;
  return cudaGetLastError();
}

}  // namespace

// One step of a state with frequency groups: float rows in the quad layout on
// a static mesh take the fused kernel (transport and source in one launch);
// the others the transport sweep, then the source step in place on I*.
cudaError_t launch_group_step(rt_state *s, double dt, const void *In, void *Out) {
  if (s->precision == RT_FP32 && s->quad_end > 0 && !s->moving && s->n_groups <= kTileGroups &&
      s->row_stride == s->n_angles) {
    switch (s->n_angles / 16) {
      case 2: return launch_fused_q<step::QuadMap<1, false>>(s, dt, In, Out);
      case 3: return launch_fused_q<step::QuadMap<1, true>>(s, dt, In, Out);
      case 4: return launch_fused_q<step::QuadMap<2, false>>(s, dt, In, Out);
      case 5: return launch_fused_q<step::QuadMap<2, true>>(s, dt, In, Out);
      case 6: return launch_fused_q<step::QuadMap<3, false>>(s, dt, In, Out);
      case 7: return launch_fused_q<step::QuadMap<3, true>>(s, dt, In, Out);
      default: return launch_fused_q<step::QuadMap<4, false>>(s, dt, In, Out);
    }
  }
  cudaError_t e = launch_transport(s, dt, In, Out, false);
  if (e == cudaSuccess) e = launch_group_source(s, dt, Out);
  return e;
}

cudaError_t launch_group_source(rt_state *s, double dt, void *Is) {
  if (s->n_groups > kMaxGroups) return cudaErrorInvalidValue;
  return s->precision == RT_FP32 ? launch<float>(s, dt, Is) : launch<double>(s, dt, Is);
}

}  // namespace rt
