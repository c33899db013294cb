// Fused radiation step: upwind transport (Sec. 3.2) + implicit comoving
// source update with gas exchange (Sec. 3.3), boundary cells (Sec. 3.5) and
// emitter cells (Sec. 3.6), one kernel per step.
//
// Mapping: KT consecutive threads own one cell; thread `sub` owns the angle
// pairs p = sub + KT*j (j < PPT) and their antipodes p + A/2, whose flux
// coefficient is u(p + A/2) = -(n_p . s) - w.  The cell's I row is read
// once, neighbour values only for the inflow side of each pair, and the
// face sum is taken in the cell's slot order (no atomics, deterministic).
// Per-cell angular sums are reduced over the KT lanes with xor shuffles.
#include <cuda_runtime.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

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

template <int KT, typename T> __device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = KT / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Positive root of alpha T^4 + beta T = g (alpha >= 0, beta > 0, g >= 0):
// Newton from above, T0 = min(g/beta, (g/alpha)^(1/4)); f is increasing and
// convex, so the iterates fall monotonically onto the root.
__device__ __forceinline__ int quartic_root(double alpha, double beta, double g, int max_iter,
                                            double *T_out) {
  double T = g / beta;
  if (alpha > 0.0) T = fmin(T, sqrt(sqrt(g / alpha)));
  bool done = false;
  int it = 0;
  while (!done && it < max_iter) {
    double T2 = T * T;
    double f = fma(alpha * T2, T2, fma(beta, T, -g));
    double fp = fma(4.0 * alpha * T2, T, beta);
    double Tn = T - f / fp;
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

template <typename R, int KT, int PPT>
__global__ void __launch_bounds__(256) step_kernel(const StepArgs<R> a) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cell = tid / KT;
  const int sub = threadIdx.x % KT;
  const bool live = cell < a.n_cells;
  const int64_t c = live ? cell : a.n_cells - 1;  // dead lanes shadow the last cell
  const int A = a.n_angles, H = a.half;

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

  // ---- transport: I* = I - dt/V sum_f u I_up
  const int64_t k0 = a.ptr[c], k1 = a.ptr[c + 1];
  for (int64_t k = k0; k < k1; ++k) {
    const int32_t nb = __ldg(a.nbr + k);
    const auto s = load_slot<R>(a.slot + k);
    const R *In = a.I_in + (size_t)nb * A;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int p = sub + KT * j;
      if (p < H) {
        const R d = fma(nx[j], s.sx, fma(ny[j], s.sy, nz[j] * s.sz));
        const R ua = d - s.w;
        const R ub = -d - s.w;
        R va = Ia[j], vb = Ib[j];
        if (ua < R(0)) va = __ldg(In + p);
        if (ub < R(0)) vb = __ldg(In + p + H);
        acca[j] = fma(ua, va, acca[j]);
        accb[j] = fma(ub, vb, accb[j]);
      }
    }
  }
  const R dtv = R(a.dt) * a.inv_vol[c];
  R wa[PPT], wb[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int p = sub + KT * j;
    const bool v = p < H;
    Ia[j] = v ? fma(-dtv, acca[j], Ia[j]) : R(0);  // now I*
    Ib[j] = v ? fma(-dtv, accb[j], Ib[j]) : R(0);
    wa[j] = v ? a.wt[p] : R(0);
    wb[j] = v ? a.wt[p + H] : R(0);
  }

  // ---- source step
  const int kind = a.kind[c];
  const GasStatic gs = a.gs[c];
  GasDyn gd = a.gd[c];
  const double inv_rho = 1.0 / gs.rho;
  const double vx = gd.mx * inv_rho, vy = gd.my * inv_rho, vz = gd.mz * inv_rho;
  const double inv_c = 1.0 / a.c;
  R Ga[PPT], Gb[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    // Gamma = 1 - v . n / c (first order in v/c); the antipode has 1 + v . n / c
    const double vn = (vx * (double)nx[j] + vy * (double)ny[j] + vz * (double)nz[j]) * inv_c;
    Ga[j] = R(1.0 - vn);
    Gb[j] = R(1.0 + vn);
  }
  // Comoving weights and the angular sums of Eq. (Jcom).  Every lane takes
  // part in the reductions whatever its cell's kind, so the shuffles below
  // are never divergent; only interior cells use the result.
  const R xs = R(a.dt * a.cbar * gs.rho * (gs.kJ + gs.kS));
  R wsum = 0, sI = 0, sG = 0;
  R Ita[PPT], Itb[PPT], xa[PPT], xb[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const R Ga2 = Ga[j] * Ga[j], Gb2 = Gb[j] * Gb[j];
    Ita[j] = Ga2 * Ga2 * Ia[j];
    Itb[j] = Gb2 * Gb2 * Ib[j];
    const R wca = wa[j] / Ga2, wcb = wb[j] / Gb2;
    xa[j] = xs * Ga[j];
    xb[j] = xs * Gb[j];
    const R ra = R(1) / (R(1) + xa[j]), rb = R(1) / (R(1) + xb[j]);
    wsum += wca + wcb;
    sI += wca * Ita[j] * ra + wcb * Itb[j] * rb;
    sG += wca * Ga[j] * ra + wcb * Gb[j] * rb;
  }
  wsum = group_sum<KT>(wsum);
  sI = group_sum<KT>(sI);
  sG = group_sum<KT>(sG);

  R In_a[PPT], In_b[PPT];
  unsigned bad = 0;
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
      In_a[j] = ((Ga4 * Ia[j] + ya * isrc) / (R(1) + ya)) / Ga4;
      In_b[j] = ((Gb4 * Ib[j] + yb * isrc) / (R(1) + yb)) / Gb4;
    }
  } else {
    const double SI = (double)sI / (double)wsum, SG = (double)sG / (double)wsum;
    const double dcr = a.dt * a.cbar * gs.rho;
    const double D = 1.0 - dcr * gs.kS * SG;
    const double rcv = gs.rho * a.rcv;
    const double kin = 0.5 * (gd.mx * gd.mx + gd.my * gd.my + gd.mz * gd.mz) * inv_rho;
    const double Tn = (gd.e - kin) / rcv;
    const double alpha = a.dt * a.c * gs.rho * gs.kP * a.a_rad * (1.0 - dcr * gs.kJ * SG / D);
    const double g = rcv * Tn + a.dt * a.c * gs.rho * 4.0 * kPi * gs.kJ * SI / D;
    double T = 0.0;
    if (!(g >= 0.0) || !(alpha >= 0.0)) {
      bad |= ST_NONFINITE;
    } else if (quartic_root(alpha, rcv, g, a.newton_max_iter, &T)) {
      bad |= ST_NONCONV;
    }
    const double B = a.a_rad * (T * T) * (T * T) / (4.0 * kPi);
    const double J = (SI + dcr * gs.kP * B * SG) / D;
    const R q = R(dcr * (gs.kP * B + gs.kS * J));
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const R Ga2 = Ga[j] * Ga[j], Gb2 = Gb[j] * Gb[j];
      In_a[j] = ((Ita[j] + q * Ga[j]) / (R(1) + xa[j])) / (Ga2 * Ga2);
      In_b[j] = ((Itb[j] + q * Gb[j]) / (R(1) + xb[j])) / (Gb2 * Gb2);
    }
  }

  // ---- store I^{n+1}; exchange from the stored values: dE = 4 pi sum w (I* - I')
  R de = 0, dfx = 0, dfy = 0, dfz = 0;
  R *Io = a.I_out + (size_t)c * A;
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int p = sub + KT * j;
    if (p < H) {
      if (live) {
        Io[p] = In_a[j];
        Io[p + H] = In_b[j];
      }
      if (!isfinite(In_a[j]) || !isfinite(In_b[j])) bad |= ST_NONFINITE;
      const R da = wa[j] * (Ia[j] - In_a[j]);
      const R db = wb[j] * (Ib[j] - In_b[j]);
      de += da + db;
      const R dd = da - db;  // antipode has direction -n
      dfx = fma(nx[j], dd, dfx);
      dfy = fma(ny[j], dd, dfy);
      dfz = fma(nz[j], dd, dfz);
    }
  }
  de = group_sum<KT>(de);
  dfx = group_sum<KT>(dfx);
  dfy = group_sum<KT>(dfy);
  dfz = group_sum<KT>(dfz);
  bad = __reduce_or_sync(0xffffffffu, bad);  // whole warp; harmless over-reporting across cells
  if (live && sub == 0) {
    const double fe = a.c / a.cbar * 4.0 * kPi * (double)de;
    const double fm = 4.0 * kPi / a.cbar;  // (4 pi c sum w n dI) / (c cbar)
    if (kind == RT_CELL_INTERIOR) {
      gd.e += fe;
      gd.mx += fm * (double)dfx;
      gd.my += fm * (double)dfy;
      gd.mz += fm * (double)dfz;
      a.gd[c] = gd;
    } else {
      double *x = a.ext + 4 * c;
      x[0] += fe;
      x[1] += fm * (double)dfx;
      x[2] += fm * (double)dfy;
      x[3] += fm * (double)dfz;
    }
    if (bad) {
      atomicOr(a.status, bad);
      atomicMin(a.bad_cell, (unsigned long long)c);
    }
  }
}

template <typename R, int KT, int PPT>
cudaError_t launch_t(rt_state *s, double dt) {
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
  a.cbar = s->params.cbar;
  a.c = s->params.c;
  a.a_rad = s->params.a_rad;
  a.rcv = s->params.r_gas / (s->params.gamma_gas - 1.0);
  a.newton_max_iter = s->params.newton_max_iter;
  a.status = s->d_status;
  a.bad_cell = s->d_bad;
  const int threads = 256;
  const int64_t total = s->n_cells * KT;
  const unsigned blocks = (unsigned)((total + threads - 1) / threads);
  step_kernel<R, KT, PPT><<<blocks, threads, 0, s->stream>>>(a);
  s->launches++;
  return cudaGetLastError();
}

template <typename R> cudaError_t dispatch(rt_state *s, double dt) {
  const int H = s->n_angles / 2;
  const int ppt = (H + 7) / 8;
  switch (ppt) {
    case 1: return launch_t<R, 8, 1>(s, dt);
    case 2: return launch_t<R, 8, 2>(s, dt);
    case 3: return launch_t<R, 8, 3>(s, dt);
    case 4: return launch_t<R, 8, 4>(s, dt);
    case 5: return launch_t<R, 8, 5>(s, dt);
    case 6: return launch_t<R, 8, 6>(s, dt);
    case 7: return launch_t<R, 8, 7>(s, dt);
    case 8: return launch_t<R, 8, 8>(s, dt);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_step(rt_state *s, double dt) {
  cudaError_t e = (s->precision == RT_FP32) ? dispatch<float>(s, dt) : dispatch<double>(s, dt);
  if (e == cudaSuccess) s->cur ^= 1;
  return e;
}

}  // namespace rt
