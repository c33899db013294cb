// Tile machinery shared by the fused step kernel (rt_step.cu) and the
// transport-only kernels (rt_transport.cu): the shared-memory stage of a
// block's face slots, the pair / quad maps of a thread's angles, and the
// face sums over a cell's slots in slot order.
#pragma once

#include <cuda_runtime.h>

#include "rt_internal.cuh"
#include "rt_step_common.cuh"

namespace rt {
namespace step {

// What a face sum accumulates: the forward upwind flux sum_f u I_up, or
// the terms sum_{f, u > 0} u (L_own - L_nbr) of the transposed transport
// operator (the adjoint, rt_adjoint.cu).
enum : int { TRANSPORT_FORWARD = 0, TRANSPORT_ADJOINT = 1 };

// One face's term of the transposed sum for one pair, the counterpart of
// face_pair: with u = d - w for angle p and u' = -d - w for its antipode and
// L = dt/V lambda per cell, acc += u (L_own - L_nbr) where u > 0 (the faces
// through which the angle leaves the cell), and the same with u' for the
// antipode.
template <typename R, bool MOVING>
__device__ __forceinline__ void face_pair_adjoint(R d, R w, R vx, R vy, R Ia, R Ib, R &acca,
                                                  R &accb) {
  if (MOVING) {
    const R ua = d - w, ub = -d - w;
    acca = fma(positive(ua) ? ua : R(0), Ia - vx, acca);
    accb = fma(positive(ub) ? ub : R(0), Ib - vy, accb);
  } else {
    // u_a = d, u_b = -d: at most one of the pair leaves through the face
    const bool out = positive(d);
    const R t = out ? Ia - vx : Ib - vy;
    acca = fma(out ? d : R(0), t, acca);
    accb = fma(out ? R(0) : -d, t, accb);
  }
}

// Gas records of a block's cells in shared memory, for the lane-per-cell
// phases (B for double states, D).
struct SharedGas {
  GasStatic gs[CPB];
  GasDyn gd[CPB];
};

// One tile's inputs staged in shared memory by the float QuadMap kernel:
// the tile's face slots (static meshes: with the neighbour index in w), the
// neighbour indices (moving meshes) and the gas records.
struct StageView {
  SlotF *slot;
  int32_t *nbr;
  SharedGas *gas;
};
__host__ __device__ inline int stage_cap(int64_t max_block_slots) {
  return (int)((max_block_slots + 7) & ~int64_t(7));
}
__host__ __device__ inline size_t stage_gas_offset(int cap, bool moving) {
  return ((size_t)cap * (sizeof(SlotF) + (moving ? sizeof(int32_t) : 0)) + 63) & ~size_t(63);
}
__host__ __device__ inline size_t stage_bytes(int cap, bool moving) {
  return stage_gas_offset(cap, moving) + sizeof(SharedGas);
}
__device__ __forceinline__ StageView stage_at(unsigned char *base, int cap, bool moving) {
  StageView v;
  v.slot = reinterpret_cast<SlotF *>(base);
  v.nbr = reinterpret_cast<int32_t *>(base + (size_t)cap * sizeof(SlotF));
  v.gas = reinterpret_cast<SharedGas *>(base + stage_gas_offset(cap, moving));
  return v;
}

// All threads: asynchronous copies of tile `tile`'s slots, neighbour indices
// and (GAS) gas records into v (one contiguous range of each array).
template <bool MOVING, bool GAS = true>
__device__ __forceinline__ void issue_stage(const StepArgs<float> &a, int64_t tile,
                                            const StageView &v) {
  const int64_t c0 = tile * CPB;
  const int64_t c1 = c0 + CPB < a.n_cells ? c0 + CPB : a.n_cells;
  const int64_t kb = a.ptr[c0];
  const int cnt = (int)(a.ptr[c1] - kb);
  if (MOVING) {
    const SlotF *gsl = reinterpret_cast<const SlotF *>(a.slot) + kb;
    for (int i = threadIdx.x; i < cnt; i += NT) {
      cp_async16(v.slot + i, gsl + i);
      cp_async4(v.nbr + i, a.nbr + kb + i);
    }
  } else {
    for (int i = threadIdx.x; i < cnt; i += NT) cp_async16(v.slot + i, a.slot_nb + kb + i);
  }
  if (!GAS) return;
  // 6 x 16 bytes per cell: GasStatic (64) then GasDyn (32)
  const int nc = (int)(c1 - c0);
  for (int i = threadIdx.x; i < 6 * nc; i += NT) {
    const int cc = i / 6, k = i % 6;
    if (k < 4)
      cp_async16(reinterpret_cast<char *>(&v.gas->gs[cc]) + 16 * k,
                 reinterpret_cast<const char *>(a.gs + c0 + cc) + 16 * k);
    else
      cp_async16(reinterpret_cast<char *>(&v.gas->gd[cc]) + 16 * (k - 4),
                 reinterpret_cast<const char *>(a.gd + c0 + cc) + 16 * (k - 4));
  }
}

// ------------------------------------------------------------ pair maps
// count(H, sub): pairs the thread owns (entries j >= count are padding);
// pair(j, sub): pair index of entry j; load / store: the thread's entries of
// one row (x = angle p, y = angle p + A/2).
template <typename R, int PPT_, bool FULL_> struct PairMap {
  static constexpr int PPT = PPT_;
  static constexpr bool FULL = FULL_;
  static constexpr bool QUAD = false;
  using V = pair_t<R>;
  __device__ static int count(int H, int sub) { return FULL ? PPT : (H - sub + KT - 1) / KT; }
  __device__ static int pair(int j, int sub) { return sub + KT * j; }
  __device__ static void load(const R *__restrict__ row, int sub, R (&x)[PPT], R (&y)[PPT],
                              int np) {
    const V *p = reinterpret_cast<const V *>(row) + sub;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const V t = (FULL || j < np) ? p[KT * j] : mk(R(0), R(0));
      x[j] = t.x;
      y[j] = t.y;
    }
  }
  __device__ static void store(R *__restrict__ row, int sub, const R (&x)[PPT],
                               const R (&y)[PPT], int np) {
    V *p = reinterpret_cast<V *>(row) + sub;
#pragma unroll
    for (int j = 0; j < PPT; ++j)
      if (FULL || j < np) p[KT * j] = mk(x[j], y[j]);
  }
};

// The quad region of a row holds (I_2Q, I_2Q+1, I_2Q+H, I_2Q+1+H) per 16 bytes
// (angle_of_position with quad_end = 32 Q4), the tail pairs side by side.
template <int Q4_, bool TAIL_> struct QuadMap {
  static constexpr int Q4 = Q4_;
  static constexpr bool TAIL = TAIL_;
  static constexpr int PPT = 2 * Q4 + (TAIL ? 1 : 0);
  static constexpr bool FULL = true;
  static constexpr bool QUAD = true;
  __device__ static int count(int, int) { return PPT; }
  __device__ static int pair(int j, int sub) {
    return j < 2 * Q4 ? 2 * (sub + KT * (j >> 1)) + (j & 1) : 16 * Q4 + sub;
  }
  __device__ static void load(const float *__restrict__ row, int sub, float (&x)[PPT],
                              float (&y)[PPT], int) {
    const float4 *q = reinterpret_cast<const float4 *>(row) + sub;
#pragma unroll
    for (int i = 0; i < Q4; ++i) {
      const float4 t = q[KT * i];
      x[2 * i] = t.x;
      x[2 * i + 1] = t.y;
      y[2 * i] = t.z;
      y[2 * i + 1] = t.w;
    }
    if (TAIL) {
      const float2 t = reinterpret_cast<const float2 *>(row)[16 * Q4 + sub];
      x[2 * Q4] = t.x;
      y[2 * Q4] = t.y;
    }
  }
  __device__ static void store(float *__restrict__ row, int sub, const float (&x)[PPT],
                               const float (&y)[PPT], int) {
    float4 *q = reinterpret_cast<float4 *>(row) + sub;
#pragma unroll
    for (int i = 0; i < Q4; ++i)
      q[KT * i] = make_float4(x[2 * i], x[2 * i + 1], y[2 * i], y[2 * i + 1]);
    if (TAIL) reinterpret_cast<float2 *>(row)[16 * Q4 + sub] = make_float2(x[2 * Q4], y[2 * Q4]);
  }
};

// face_sum for QuadMap (float): the two pairs of a quad are processed as
// f32x2 vectors.  Per face and pair, with d = n . s and u = d - w for the
// angle, u' = -d - w for its antipode:
//   acc  += max(u, 0) I_own + min(u, 0) I_nbr          (upwind value of u)
//   acc' += min(e, 0) I'_own + max(e, 0) I'_nbr,  e = d + w = -u',
// and the antipode's sum is -acc'.  One of each max / min is zero, so this
// equals the select-and-multiply form exactly.  MODE TRANSPORT_ADJOINT sums
// the transposed operator's terms instead (face_pair_adjoint):
//   acc  += max(u, 0) (L_own - L_nbr),  acc' += min(e, 0) (L'_own - L'_nbr).
template <typename M, bool MOVING, bool PACKED, int MODE, typename K>
__device__ __forceinline__ void face_sum_quads(const SlotF *__restrict__ slot,
                                               const int32_t *__restrict__ nbr, K k0, K k1,
                                               const float *__restrict__ I_in, int RS, int sub,
                                               const float (&nx)[M::PPT], const float (&ny)[M::PPT],
                                               const float (&nz)[M::PPT], const float (&Ia)[M::PPT],
                                               const float (&Ib)[M::PPT], float (&acca)[M::PPT],
                                               float (&accb)[M::PPT]) {
  constexpr int Q4 = M::Q4;
  float2 NX[Q4], NY[Q4], NZ[Q4], OA[Q4], OB[Q4], CA[Q4], CB[Q4];
#pragma unroll
  for (int i = 0; i < Q4; ++i) {
    NX[i] = make_float2(nx[2 * i], nx[2 * i + 1]);
    NY[i] = make_float2(ny[2 * i], ny[2 * i + 1]);
    NZ[i] = make_float2(nz[2 * i], nz[2 * i + 1]);
    OA[i] = make_float2(Ia[2 * i], Ia[2 * i + 1]);
    OB[i] = make_float2(Ib[2 * i], Ib[2 * i + 1]);
    CA[i] = make_float2(0.0f, 0.0f);
    CB[i] = CA[i];
  }
  const float2 zero = make_float2(0.0f, 0.0f);
#pragma unroll 2
  for (K k = k0; k < k1; ++k) {
    const float4 s = *reinterpret_cast<const float4 *>(slot + k);
    int32_t nb;
    if constexpr (PACKED)
      nb = __float_as_int(s.w);
    else
      nb = nbr[k];
    const float *row = I_in + (size_t)nb * RS;
    const float4 *q = reinterpret_cast<const float4 *>(row) + sub;
    float4 v[Q4];
#pragma unroll
    for (int i = 0; i < Q4; ++i) v[i] = q[KT * i];
    float2 vt = zero;
    if (M::TAIL) vt = reinterpret_cast<const float2 *>(row)[16 * Q4 + sub];
    const float2 SX = make_float2(s.x, s.x), SY = make_float2(s.y, s.y),
                 SZ = make_float2(s.z, s.z);
    const float w = MOVING ? s.w : 0.0f;
    const float2 W = make_float2(w, w);
#pragma unroll
    for (int i = 0; i < Q4; ++i) {
      const float2 D = pfma(NX[i], SX, pfma(NY[i], SY, pmul(NZ[i], SZ)));
      const float2 U = MOVING ? psub(D, W) : D;   // u of the two angles
      const float2 E = MOVING ? padd(D, W) : D;   // -u' of their antipodes
      const float2 UP = make_float2(fmaxf(U.x, 0.0f), fmaxf(U.y, 0.0f));
      const float2 EM = MOVING ? make_float2(fminf(E.x, 0.0f), fminf(E.y, 0.0f))
                               : make_float2(fminf(U.x, 0.0f), fminf(U.y, 0.0f));
      if constexpr (MODE == TRANSPORT_FORWARD) {
        const float2 UM = MOVING ? make_float2(fminf(U.x, 0.0f), fminf(U.y, 0.0f)) : EM;
        const float2 EP = MOVING ? make_float2(fmaxf(E.x, 0.0f), fmaxf(E.y, 0.0f)) : UP;
        CA[i] = pfma(UP, OA[i], pfma(UM, make_float2(v[i].x, v[i].y), CA[i]));
        CB[i] = pfma(EM, OB[i], pfma(EP, make_float2(v[i].z, v[i].w), CB[i]));
      } else {
        CA[i] = pfma(UP, psub(OA[i], make_float2(v[i].x, v[i].y)), CA[i]);
        CB[i] = pfma(EM, psub(OB[i], make_float2(v[i].z, v[i].w)), CB[i]);
      }
    }
    if (M::TAIL) {
      constexpr int j = 2 * Q4;
      const float d = fmaf(nx[j], s.x, fmaf(ny[j], s.y, nz[j] * s.z));
      if constexpr (MODE == TRANSPORT_FORWARD)
        face_pair<float, MOVING>(d, w, vt.x, vt.y, Ia[j], Ib[j], acca[j], accb[j]);
      else
        face_pair_adjoint<float, MOVING>(d, w, vt.x, vt.y, Ia[j], Ib[j], acca[j], accb[j]);
    }
  }
#pragma unroll
  for (int i = 0; i < Q4; ++i) {
    acca[2 * i] = CA[i].x;
    acca[2 * i + 1] = CA[i].y;
    accb[2 * i] = -CB[i].x;
    accb[2 * i + 1] = -CB[i].y;
  }
}

// sum_f u I_up over the slots [k0, k1) of one cell, neighbour rows read
// through nbr[k] (L1/L2 serve the reuse between neighbouring cells; cells are
// in Morton order).  slot / nbr point either to global memory or to the
// block's copy in shared memory (K = int); PACKED: static float slots carry
// the neighbour index in their w word and nbr is not read.
template <typename R, typename M, bool MOVING, bool PACKED, int MODE, typename S, typename K>
__device__ __forceinline__ void face_sum(const S *__restrict__ slot, const int32_t *__restrict__ nbr,
                                         const double *__restrict__ wface,
                                         const double *__restrict__ uface, int H, K k0, K k1,
                                         const R *__restrict__ I_in, int RS, int sub,
                                         const R (&nx)[M::PPT], const R (&ny)[M::PPT],
                                         const R (&nz)[M::PPT], const R (&Ia)[M::PPT],
                                         const R (&Ib)[M::PPT], R (&acca)[M::PPT],
                                         R (&accb)[M::PPT], int np) {
  constexpr int PPT = M::PPT;
  if constexpr (M::QUAD) {
    face_sum_quads<M, MOVING, PACKED, MODE>(slot, nbr, k0, k1, I_in, RS, sub, nx, ny, nz, Ia, Ib,
                                            acca, accb);
  } else {
#pragma unroll 2
    for (K k = k0; k < k1; ++k) {
      const S s = slot[k];
      int32_t nb;
      if constexpr (PACKED)
        nb = __float_as_int(s.w);
      else
        nb = nbr[k];
      R vx[PPT], vy[PPT];
      M::load(I_in + (size_t)nb * RS, sub, vx, vy, np);
      const R w = MOVING ? slot_w(s, wface, k) : R(0);
#pragma unroll
      for (int j = 0; j < PPT; ++j)
        if (M::FULL || j < np) {
          R d;
          if constexpr (sizeof(R) == 8)
            d = uface[(size_t)k * H + M::pair(j, sub)];  // the table built by build_uface
          else
            d = slot_dot(nx[j], ny[j], nz[j], s);
          if constexpr (MODE == TRANSPORT_FORWARD)
            face_pair<R, MOVING>(d, w, vx[j], vy[j], Ia[j], Ib[j], acca[j], accb[j]);
          else
            face_pair_adjoint<R, MOVING>(d, w, vx[j], vy[j], Ia[j], Ib[j], acca[j], accb[j]);
        }
    }
  }
}


}  // namespace step
}  // namespace rt
