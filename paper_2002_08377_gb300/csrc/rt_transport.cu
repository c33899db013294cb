// Transport-only sweeps on the step kernel's tile machinery (the same
// blocks of 32 cells x 8 threads, pair / quad maps, shared-memory stage and
// face order), the building blocks of the discrete adjoint (rt_adjoint.cu):
//   TRANSPORT_FORWARD  I* = I - dt/V_c sum_f u I_up                 (Sec. 2.2)
//   TRANSPORT_ADJOINT  (M^T lambda)_c = lambda_c - sum_{f, u > 0} u (L_c - L_nbr)
//                      with the input rows L = dt/V lambda (per cell), written
//                      as L_c V_c/dt - sum.
// No source step and no gas.
#include <cuda_runtime.h>

#include "rt_internal.cuh"
#include "rt_step_common.cuh"
#include "rt_step_tile.cuh"

namespace rt {
namespace {
using namespace step;

template <typename R, typename M, bool MOVING, bool STAGED, int MODE>
__device__ __forceinline__ void tile_transport(const StepArgs<R> &a, const int64_t tile,
                                               const StageView &stage) {
  constexpr int PPT = M::PPT;
  const int lc = threadIdx.x / KT;
  const int sub = threadIdx.x % KT;
  const int64_t cell = tile * CPB + lc;
  const bool live = cell < a.n_cells;
  const int64_t c = live ? cell : a.n_cells - 1;  // dead lanes shadow the last cell
  const int RS = a.row;
  const int np = M::count(a.half, sub);
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
    face_sum<R, M, MOVING, !MOVING, MODE>(
        reinterpret_cast<const typename SlotOf<R>::type *>(stage.slot), stage.nbr, a.wface,
        a.uface, a.half, k0, k1, a.I_in, RS, sub, nx, ny, nz, Ia, Ib, acca, accb, np);
  } else {
    face_sum<R, M, MOVING, false, MODE>(a.slot, a.nbr, a.wface, a.uface, a.half, a.ptr[c],
                                        a.ptr[c + 1], a.I_in, RS, sub, nx, ny, nz, Ia, Ib, acca,
                                        accb, np);
  }
  const R dtv = a.dt_r * a.inv_vol[c];
  if constexpr (MODE == TRANSPORT_FORWARD) {
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      Ia[j] = fma(-dtv, acca[j], Ia[j]);
      Ib[j] = fma(-dtv, accb[j], Ib[j]);
    }
  } else {
    const R vdt = rcp(dtv);
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      Ia[j] = fma(Ia[j], vdt, -acca[j]);
      Ib[j] = fma(Ib[j], vdt, -accb[j]);
    }
  }
  if (live) M::store(a.I_out + (size_t)c * RS, sub, Ia, Ib, np);
}

template <typename R, int PPT> constexpr int min_blocks() {
  return (sizeof(R) == 4 ? (PPT <= 5 ? 1024 : 768) : 512) / NT;
}

template <typename R, typename M, bool MOVING, int MODE>
__global__ void __launch_bounds__(NT, min_blocks<R, M::PPT>())
    transport_kernel(const StepArgs<R> a) {
  tile_transport<R, M, MOVING, false, MODE>(a, blockIdx.x, StageView{});
}

// Float rows in the quad layout: the block's slots (and, moving meshes, the
// neighbour indices) are first copied into shared memory.
template <typename M, bool MOVING, int MODE>
__global__ void __launch_bounds__(NT, min_blocks<float, M::PPT>())
    transport_kernel_staged(const StepArgs<float> a, int cap) {
  extern __shared__ __align__(128) unsigned char dyn[];
  const StageView v = stage_at(dyn, cap, MOVING);
  issue_stage<MOVING, false>(a, blockIdx.x, v);
  tile_transport<float, M, MOVING, true, MODE>(a, blockIdx.x, v);
}

template <typename R, typename M, bool MOVING, bool STAGED, int MODE>
cudaError_t launch_tr(rt_state *s, double dt, const void *in, void *out) {
  StepArgs<R> a{};
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
  a.dir = reinterpret_cast<const R *>(s->d_dir);
  a.I_in = reinterpret_cast<const R *>(in);
  a.I_out = reinterpret_cast<R *>(out);
  a.dt = dt;
  a.dt_r = R(dt);
  const unsigned blocks = (unsigned)((s->n_cells + CPB - 1) / CPB);
  if constexpr (STAGED) {
    const int cap = stage_cap(s->max_block_slots);
    transport_kernel_staged<M, MOVING, MODE>
        <<<blocks, NT, stage_gas_offset(cap, MOVING), s->stream>>>(a, cap);
  } else {
    transport_kernel<R, M, MOVING, MODE><<<blocks, NT, 0, s->stream>>>(a);
  }
  s->launches++;
  return cudaGetLastError();
}

template <typename R, bool MOVING, bool FULL, int MODE>
cudaError_t dispatch_pairs(rt_state *s, double dt, const void *in, void *out) {
  switch ((s->n_angles / 2 + KT - 1) / KT) {
    case 1: return launch_tr<R, PairMap<R, 1, FULL>, MOVING, false, MODE>(s, dt, in, out);
    case 2: return launch_tr<R, PairMap<R, 2, FULL>, MOVING, false, MODE>(s, dt, in, out);
    case 3: return launch_tr<R, PairMap<R, 3, FULL>, MOVING, false, MODE>(s, dt, in, out);
    case 4: return launch_tr<R, PairMap<R, 4, FULL>, MOVING, false, MODE>(s, dt, in, out);
    case 5: return launch_tr<R, PairMap<R, 5, FULL>, MOVING, false, MODE>(s, dt, in, out);
    case 6: return launch_tr<R, PairMap<R, 6, FULL>, MOVING, false, MODE>(s, dt, in, out);
    case 7: return launch_tr<R, PairMap<R, 7, FULL>, MOVING, false, MODE>(s, dt, in, out);
    case 8: return launch_tr<R, PairMap<R, 8, FULL>, MOVING, false, MODE>(s, dt, in, out);
    default: return cudaErrorInvalidValue;
  }
}

template <bool MOVING, int MODE>
cudaError_t dispatch_quads(rt_state *s, double dt, const void *in, void *out) {
  switch (s->n_angles / 16) {
    case 2: return launch_tr<float, QuadMap<1, false>, MOVING, true, MODE>(s, dt, in, out);
    case 3: return launch_tr<float, QuadMap<1, true>, MOVING, true, MODE>(s, dt, in, out);
    case 4: return launch_tr<float, QuadMap<2, false>, MOVING, true, MODE>(s, dt, in, out);
    case 5: return launch_tr<float, QuadMap<2, true>, MOVING, true, MODE>(s, dt, in, out);
    case 6: return launch_tr<float, QuadMap<3, false>, MOVING, true, MODE>(s, dt, in, out);
    case 7: return launch_tr<float, QuadMap<3, true>, MOVING, true, MODE>(s, dt, in, out);
    case 8: return launch_tr<float, QuadMap<4, false>, MOVING, true, MODE>(s, dt, in, out);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, int MODE>
cudaError_t dispatch(rt_state *s, double dt, const void *in, void *out) {
  if (sizeof(R) == 4 && s->quad_end > 0)  // rows in the quad layout
    return s->moving ? dispatch_quads<true, MODE>(s, dt, in, out)
                     : dispatch_quads<false, MODE>(s, dt, in, out);
  const bool full = (s->n_angles / 2) % KT == 0;
  if (s->moving)
    return full ? dispatch_pairs<R, true, true, MODE>(s, dt, in, out)
                : dispatch_pairs<R, true, false, MODE>(s, dt, in, out);
  return full ? dispatch_pairs<R, false, true, MODE>(s, dt, in, out)
              : dispatch_pairs<R, false, false, MODE>(s, dt, in, out);
}

}  // namespace

cudaError_t launch_transport(rt_state *s, double dt, const void *in, void *out, bool adjoint) {
  if (s->precision == RT_FP32)
    return adjoint ? dispatch<float, TRANSPORT_ADJOINT>(s, dt, in, out)
                   : dispatch<float, TRANSPORT_FORWARD>(s, dt, in, out);
  return adjoint ? dispatch<double, TRANSPORT_ADJOINT>(s, dt, in, out)
                 : dispatch<double, TRANSPORT_FORWARD>(s, dt, in, out);
}

}  // namespace rt
