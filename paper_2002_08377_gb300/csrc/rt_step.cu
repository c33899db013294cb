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
#include "rt_step_common.cuh"

namespace rt {
namespace {
using namespace step;

template <typename R> struct Shared {
  GasStatic gs[CPB];  // gas of the block's cells, prefetched for warp 0
  GasDyn gd[CPB];
  R sI[CPB], sG[CPB], s1[CPB];  // the sums of Eq. (Jcom) and sum w~/(1+x), unnormalised
  R q[CPB];                     // dt cbar rho (kP B + kS J) per interior cell
  R dE[CPB], dF[3][CPB];        // sum w (I* - I') and sum w n (I* - I')
  unsigned bad[CPB];
};

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

// The same sum with the tile's neighbour rows, slots and tile-local rows
// staged in shared memory (rows `stride` bytes apart).
template <typename R, int PPT, bool MOVING, bool FULL, typename S>
__device__ __forceinline__ void face_sum_staged(const S *slot, const uint16_t *loc,
                                                const double *__restrict__ wface, int k0, int k1,
                                                const unsigned char *rows, int stride, int sub,
                                                const R (&nx)[PPT], const R (&ny)[PPT],
                                                const R (&nz)[PPT], const R (&Ia)[PPT],
                                                const R (&Ib)[PPT], R (&acca)[PPT], R (&accb)[PPT],
                                                int np) {
  using V = pair_t<R>;
#pragma unroll 4
  for (int k = k0; k < k1; ++k) {
    const S s = slot[k];
    const V *In = reinterpret_cast<const V *>(rows + (int)loc[k] * stride) + sub;
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

// A tile staged in shared memory: its own rows (0..CPB-1) and halo rows,
// its face slots and their tile-local rows; rows == nullptr: global path.
template <typename R> struct TileStage {
  const unsigned char *rows = nullptr;
  int stride = 0;
  const typename SlotOf<R>::type *slots = nullptr;
  const uint16_t *loc = nullptr;
};

// One tile of CPB cells: phases A-D (see the top of the file).  Ends with
// warp 0 in phase D; callers that reuse `sh` synchronise first.
template <typename R, int PPT, bool MOVING, bool FULL>
__device__ __forceinline__ void tile_step(const StepArgs<R> &a, const int64_t tile, Shared<R> &sh,
                                          const TileStage<R> stg, const unsigned timeout) {
  using V = pair_t<R>;
  const int lc = threadIdx.x / KT;
  const int sub = threadIdx.x % KT;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t cell = tile * CPB + lc;
  const bool live = cell < a.n_cells;
  const int64_t c = live ? cell : a.n_cells - 1;  // dead lanes shadow the last cell
  const int A = a.n_angles, H = a.half;
  const int np = FULL ? PPT : (H - sub + KT - 1) / KT;  // pairs p = sub + KT j < H

  // warp 0 prefetches its cells' gas state for phases B and D
  const int64_t cl = tile * CPB + lane;  // warp 0: lane-per-cell
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
    const V *Ic = stg.rows ? reinterpret_cast<const V *>(stg.rows + lc * stg.stride) + sub
                           : reinterpret_cast<const V *>(a.I_in + (size_t)c * A) + sub;
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
  if (stg.rows) {
    const int64_t kb = a.ptr[tile * CPB];
    face_sum_staged<R, PPT, MOVING, FULL>(stg.slots, stg.loc, a.wface ? a.wface + kb : nullptr,
                                          (int)(a.ptr[c] - kb), (int)(a.ptr[c + 1] - kb), stg.rows,
                                          stg.stride, sub, nx, ny, nz, Ia, Ib, acca, accb, np);
  } else {
    face_sum<R, PPT, MOVING, FULL>(a.slot, a.nbr, a.wface, a.ptr[c], a.ptr[c + 1], a.I_in, A, sub,
                                   nx, ny, nz, Ia, Ib, acca, accb, np);
  }
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
  nonfinite = cell_or(nonfinite) | timeout;
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
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 4 : 2) step_kernel(const StepArgs<R> a) {
  __shared__ Shared<R> sh;
  tile_step<R, PPT, MOVING, FULL>(a, blockIdx.x, sh, TileStage<R>{}, 0u);
}

// ------------------------------------------------------------ pipelined float kernel
// Persistent CTAs walk the tiles; while a CTA computes tile t, warp 0 has
// already asked the TMA engine for tile t + gridDim.x: its own and halo
// intensity rows, its face slots and their tile-local rows, one bulk copy
// each, into the other of two shared-memory stages, completed on that
// stage's mbarrier.  Tiles whose halo or slots exceed a stage take the
// global-gather path.
struct PipeArgs {
  int64_t n_tiles;
  const int64_t *halo_ptr;
  const int32_t *halo;
  const int64_t *loc_off;
  const uint16_t *loc;
  const uint8_t *fits;
  int stride;        // bytes per staged row (A floats)
  int stage_bytes;
  int slot_off, loc_off_b;  // byte offsets inside a stage
};

__host__ __device__ inline int pipe_slot_off(int stride) {
  return (PIPE_ROWS * stride + 127) & ~127;
}
__host__ __device__ inline int pipe_loc_off(int stride) {
  return pipe_slot_off(stride) + PIPE_SLOTS * (int)sizeof(SlotF);
}
__host__ __device__ inline int pipe_stage_bytes(int stride) {
  return (pipe_loc_off(stride) + PIPE_SLOTS * (int)sizeof(uint16_t) + 127) & ~127;
}

struct PipeShared {
  Shared<float> sh;
  unsigned long long bar[2];
};

// Issue the bulk copies of tile t into stage st (warp 0; the tile fits).
__device__ __forceinline__ void issue_tile(const StepArgs<float> &a, const PipeArgs &p, int64_t t,
                                           unsigned char *stage, unsigned long long *bar, int lane) {
  const int64_t c0 = t * CPB;
  const int64_t c1 = c0 + CPB < a.n_cells ? c0 + CPB : a.n_cells;
  const int64_t kb = a.ptr[c0];
  const unsigned cnt = (unsigned)(a.ptr[c1] - kb);
  const int64_t h0 = p.halo_ptr[t];
  const int nh = (int)(p.halo_ptr[t + 1] - h0);
  const int nown = (int)(c1 - c0);
  const unsigned rb = (unsigned)(a.n_angles * sizeof(float));
  const unsigned lb = (unsigned)((p.loc_off[t + 1] - p.loc_off[t]) * sizeof(uint16_t));
  if (lane == 0) {
    // the stage was read by the generic proxy in an earlier tile
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, rb * (unsigned)(nown + nh) + cnt * (unsigned)sizeof(SlotF) + lb);
    if (cnt > 0) {
      bulk_copy_g2s(stage + p.slot_off, a.slot + kb, cnt * (unsigned)sizeof(SlotF), bar);
      bulk_copy_g2s(stage + p.loc_off_b, p.loc + p.loc_off[t], lb, bar);
    }
  }
  __syncwarp();
  for (int r = lane; r < nown; r += 32)
    bulk_copy_g2s(stage + r * p.stride, a.I_in + (size_t)(c0 + r) * a.n_angles, rb, bar);
  for (int h = lane; h < nh; h += 32)
    bulk_copy_g2s(stage + (CPB + h) * p.stride, a.I_in + (size_t)p.halo[h0 + h] * a.n_angles, rb,
                  bar);
}

template <int PPT, bool MOVING, bool FULL>
__global__ void __launch_bounds__(NT, 2) step_kernel_pipe(const StepArgs<float> a,
                                                          const PipeArgs p) {
  __shared__ PipeShared ps;
  extern __shared__ __align__(128) unsigned char dyn[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    mbar_init(&ps.bar[0], 1);
    mbar_init(&ps.bar[1], 1);
  }
  __syncthreads();
  unsigned phase = 0;       // bit s: parity of stage s's next completion
  unsigned failed = 0;      // a bounded wait gave up: stop staging
  int64_t t = blockIdx.x;
  if (warp == 0 && t < p.n_tiles && p.fits[t]) issue_tile(a, p, t, dyn, &ps.bar[0], lane);
  for (int it = 0; t < p.n_tiles; t += gridDim.x, ++it) {
    const int st = it & 1;
    unsigned char *stage = dyn + st * p.stage_bytes;
    const int64_t tn = t + gridDim.x;
    if (warp == 0 && !failed && tn < p.n_tiles && p.fits[tn])
      issue_tile(a, p, tn, dyn + (st ^ 1) * p.stage_bytes, &ps.bar[st ^ 1], lane);
    TileStage<float> stg;
    unsigned timeout = 0;
    if (p.fits[t] && !failed) {
      if (!mbar_wait_bounded(&ps.bar[st], (phase >> st) & 1u)) {
        timeout = ST_TIMEOUT;
        failed = 1;
      }
      phase ^= 1u << st;
      if (!timeout) {
        stg.rows = stage;
        stg.stride = p.stride;
        stg.slots = reinterpret_cast<const SlotF *>(stage + p.slot_off);
        stg.loc = reinterpret_cast<const uint16_t *>(stage + p.loc_off_b);
      }
    }
    failed = __syncthreads_or(failed);
    tile_step<float, PPT, MOVING, FULL>(a, t, ps.sh, stg, timeout);
    __syncthreads();  // `sh` and this stage are reused next
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
  if constexpr (sizeof(R) == 4) {
    if (s->pipe) {
      PipeArgs p;
      p.n_tiles = s->n_tiles;
      p.halo_ptr = s->d_halo_ptr;
      p.halo = s->d_halo;
      p.loc_off = s->d_loc_off;
      p.loc = s->d_loc;
      p.fits = s->d_fits;
      p.stride = s->n_angles * (int)sizeof(float);
      p.stage_bytes = pipe_stage_bytes(p.stride);
      p.slot_off = pipe_slot_off(p.stride);
      p.loc_off_b = pipe_loc_off(p.stride);
      const size_t dyn = 2 * (size_t)p.stage_bytes;
      static bool attr_set = false;  // one per kernel instantiation
      if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel_pipe<PPT, MOVING, FULL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)dyn);
        if (e != cudaSuccess) return e;
        attr_set = true;
      }
      const int64_t want = 2 * (int64_t)s->num_sms;
      const unsigned grid = (unsigned)(s->n_tiles < want ? s->n_tiles : want);
      step_kernel_pipe<PPT, MOVING, FULL><<<grid, NT, dyn, s->stream>>>(a, p);
      s->launches++;
      return cudaGetLastError();
    }
  }
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
