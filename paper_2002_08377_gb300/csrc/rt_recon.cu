// Limited linear reconstruction and the van Leer step (Sec. 2, integration
// steps with the van Leer half step; Sec. 2.2, transport step 2: the face
// state by linear reconstruction with a limiter).
//
// One step of the van Leer integrator is four launches:
//   1. the fused step kernel over dt/2 from I^n into I^{n+1/2} (first-order
//      upwinding), its gas update discarded;
//   2. the gradient (gradient_quad for float rows in the quad layout,
//      gradient_tile otherwise): least-squares gradients of I^{n+1/2} over
//      each cell's face neighbours, weights A_f / |r_f|^2, limited
//      (Barth-Jespersen) so that the reconstructed face values stay within
//      the range of the cell and its neighbours;
//   3. the reconstructed transport (recon_transport_quad /
//      recon_transport_tile): I* = I^n - dt/V sum_f u I_up with the upwind
//      value reconstructed at the face centre from I^{n+1/2} and its gradient
//      (the same value on both sides of a face, so the update conserves);
//   4. the fused step kernel in source-only mode over dt from the gas at n.
// The paper defers the gradient estimate and the limiter to its hydro code;
// these are the readings the oracle uses too.
#include <cuda_runtime.h>

#include "rt_internal.cuh"
#include "rt_step_common.cuh"
#include "rt_step_tile.cuh"

namespace rt {
namespace {
using namespace step;

__device__ __forceinline__ float rmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double rmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float rmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double rmax(double a, double b) { return fmax(a, b); }

// Arguments of the two middle kernels of the van Leer step.
template <typename R> struct VLArgs {
  int64_t n;
  int H, RS;
  const int64_t *ptr;
  const int32_t *nbr;
  const SlotF *slotf;   // float states: (cbar A n_f, A w . n_f)
  const double *uface;  // double states: [nnz][A/2] n_p . s
  const double *wface;  // double states: A w . n_f (moving meshes)
  const R *recon;       // [nnz][8] (x_f - x_c, w_f, x_f - x_nbr', 0)
  const R *lsq;         // [N][8] inverse of sum_f w_f r_f r_f^T (xx, xy, xz, yy, yz, zz)
  const R *dir;         // [A][4]
  const R *inv_vol;
  const R *I;           // I^n
  const R *Ih;          // I^{n+1/2}
  R *G;                 // [3][N][RS] limited gradient rows (x, y, z), row layout of I
  R *Istar;
  R dt;
};

// All kernels use the step kernel's tile mapping: blocks of 32 cells x 8
// threads, faces in slot order.  Rows in the pair layout (double, and float
// rows outside the quad layout): thread `sub` owns entries j < PPT of its
// pair map (pair M::pair(j, sub) = angle p and its antipode p + A/2),
// processed in chunks [J0, J1) so that the per-entry registers of one chunk
// fit; a chunk walks the cell's faces once more.

// Entries [J0, J1) of one row in the pair layout (x = angle p, y = antipode).
template <typename M, int J0, int J1, typename R>
__device__ __forceinline__ void load_entries(const R *__restrict__ row, int sub, R (&x)[M::PPT],
                                             R (&y)[M::PPT], int np) {
  const pair_t<R> *p = reinterpret_cast<const pair_t<R> *>(row) + sub;
#pragma unroll
  for (int j = J0; j < J1; ++j) {
    const pair_t<R> t = (M::FULL || j < np) ? p[KT * j] : mk(R(0), R(0));
    x[j] = t.x;
    y[j] = t.y;
  }
}
template <typename M, int J0, int J1, typename R>
__device__ __forceinline__ void store_entries(R *__restrict__ row, int sub, const R (&x)[M::PPT],
                                              const R (&y)[M::PPT], int np) {
  pair_t<R> *p = reinterpret_cast<pair_t<R> *>(row) + sub;
#pragma unroll
  for (int j = J0; j < J1; ++j)
    if (M::FULL || j < np) p[KT * j] = mk(x[j], y[j]);
}

// Reconstruction geometry of slot k: o = x_f - x_c, r = x_f - x_nbr'
// (periodic image), w = A_f / |r_f|^2.
template <typename R> struct Geo {
  R ox, oy, oz, w, rx, ry, rz;
};
__device__ __forceinline__ Geo<float> load_geo(const float *g) {
  const float4 a = __ldg(reinterpret_cast<const float4 *>(g));
  const float4 b = __ldg(reinterpret_cast<const float4 *>(g) + 1);
  return {a.x, a.y, a.z, a.w, b.x, b.y, b.z};
}
__device__ __forceinline__ Geo<double> load_geo(const double *g) {
  const double2 *q = reinterpret_cast<const double2 *>(g);
  const double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
  return {a.x, a.y, b.x, b.y, c.x, c.y, __ldg(g + 6)};
}

// The chunk boundaries: [J0, min(J0 + CJ, PPT)), CJ even for the quad map.
template <typename M, int CJ, int J0> __host__ __device__ constexpr int chunk_end() {
  return J0 + CJ < M::PPT ? J0 + CJ : M::PPT;
}

// Gradient of entries [J0, J1): least-squares gradients of the stage-1
// intensity over the face neighbours (weights w_f, the inverse normal matrix
// in lsq), limited by the oracle's Barth-Jespersen factor min over faces of
// (max - I_c) / d_f (d_f > 0) and (min - I_c) / d_f (d_f < 0), taken as one
// division by the largest and one by the smallest d_f: correctly rounded
// division is monotone in d_f, so the result is the same number.
template <typename R, typename M, int J0, int J1>
__device__ __forceinline__ void gradient_chunk(const VLArgs<R> &a, int64_t c, int sub, int np) {
  constexpr int PPT = M::PPT;
  const int64_t k0 = a.ptr[c], k1 = a.ptr[c + 1];
  R Ia[PPT], Ib[PPT], bxa[PPT], bya[PPT], bza[PPT], bxb[PPT], byb[PPT], bzb[PPT];
  R loa[PPT], hia[PPT], lob[PPT], hib[PPT];
  load_entries<M, J0, J1>(a.Ih + (size_t)c * a.RS, sub, Ia, Ib, np);
#pragma unroll
  for (int j = J0; j < J1; ++j) {
    bxa[j] = bya[j] = bza[j] = bxb[j] = byb[j] = bzb[j] = R(0);
    loa[j] = hia[j] = Ia[j];
    lob[j] = hib[j] = Ib[j];
  }
  for (int64_t k = k0; k < k1; ++k) {
    const Geo<R> g = load_geo(a.recon + 8 * k);
    const R rx = g.ox - g.rx, ry = g.oy - g.ry, rz = g.oz - g.rz;
    R va[PPT], vb[PPT];
    load_entries<M, J0, J1>(a.Ih + (size_t)a.nbr[k] * a.RS, sub, va, vb, np);
#pragma unroll
    for (int j = J0; j < J1; ++j) {
      const R da = va[j] - Ia[j], db = vb[j] - Ib[j];
      bxa[j] += g.w * rx * da;
      bya[j] += g.w * ry * da;
      bza[j] += g.w * rz * da;
      bxb[j] += g.w * rx * db;
      byb[j] += g.w * ry * db;
      bzb[j] += g.w * rz * db;
      loa[j] = rmin(loa[j], va[j]);
      hia[j] = rmax(hia[j], va[j]);
      lob[j] = rmin(lob[j], vb[j]);
      hib[j] = rmax(hib[j], vb[j]);
    }
  }
  const R *L = a.lsq + 8 * c;
  const R m00 = L[0], m01 = L[1], m02 = L[2], m11 = L[3], m12 = L[4], m22 = L[5];
  R gxa[PPT], gya[PPT], gza[PPT], gxb[PPT], gyb[PPT], gzb[PPT];
  R xa[PPT], na[PPT], xb[PPT], nb[PPT];  // largest and smallest d_f per angle
#pragma unroll
  for (int j = J0; j < J1; ++j) {
    gxa[j] = m00 * bxa[j] + m01 * bya[j] + m02 * bza[j];
    gya[j] = m01 * bxa[j] + m11 * bya[j] + m12 * bza[j];
    gza[j] = m02 * bxa[j] + m12 * bya[j] + m22 * bza[j];
    gxb[j] = m00 * bxb[j] + m01 * byb[j] + m02 * bzb[j];
    gyb[j] = m01 * bxb[j] + m11 * byb[j] + m12 * bzb[j];
    gzb[j] = m02 * bxb[j] + m12 * byb[j] + m22 * bzb[j];
    xa[j] = na[j] = xb[j] = nb[j] = R(0);
  }
  for (int64_t k = k0; k < k1; ++k) {
    const Geo<R> g = load_geo(a.recon + 8 * k);
#pragma unroll
    for (int j = J0; j < J1; ++j) {
      const R dA = gxa[j] * g.ox + gya[j] * g.oy + gza[j] * g.oz;
      const R dB = gxb[j] * g.ox + gyb[j] * g.oy + gzb[j] * g.oz;
      xa[j] = rmax(xa[j], dA);
      na[j] = rmin(na[j], dA);
      xb[j] = rmax(xb[j], dB);
      nb[j] = rmin(nb[j], dB);
    }
  }
#pragma unroll
  for (int j = J0; j < J1; ++j) {
    R fa = 1, fb = 1;
    if (xa[j] > R(0)) fa = rmin(fa, (hia[j] - Ia[j]) / xa[j]);
    if (na[j] < R(0)) fa = rmin(fa, (loa[j] - Ia[j]) / na[j]);
    if (xb[j] > R(0)) fb = rmin(fb, (hib[j] - Ib[j]) / xb[j]);
    if (nb[j] < R(0)) fb = rmin(fb, (lob[j] - Ib[j]) / nb[j]);
    gxa[j] *= fa;
    gya[j] *= fa;
    gza[j] *= fa;
    gxb[j] *= fb;
    gyb[j] *= fb;
    gzb[j] *= fb;
  }
  const size_t plane = (size_t)a.n * a.RS, off = (size_t)c * a.RS;
  store_entries<M, J0, J1>(a.G + off, sub, gxa, gxb, np);
  store_entries<M, J0, J1>(a.G + plane + off, sub, gya, gyb, np);
  store_entries<M, J0, J1>(a.G + 2 * plane + off, sub, gza, gzb, np);
}

template <typename R, typename M, int CJ, int J0>
__device__ __forceinline__ void gradient_chunks(const VLArgs<R> &a, int64_t c, int sub, int np) {
  if constexpr (J0 < M::PPT) {
    constexpr int J1 = chunk_end<M, CJ, J0>();
    gradient_chunk<R, M, J0, J1>(a, c, sub, np);
    gradient_chunks<R, M, CJ, J1>(a, c, sub, np);
  }
}

template <typename R, typename M, int CJ>
__global__ void __launch_bounds__(NT, 2) gradient_tile(const VLArgs<R> a) {
  const int lc = threadIdx.x / KT, sub = threadIdx.x % KT;
  const int64_t c = (int64_t)blockIdx.x * CPB + lc;
  if (c >= a.n) return;  // no barrier below
  gradient_chunks<R, M, CJ, 0>(a, c, sub, M::count(a.H, sub));
}

// sum_f u I_up for entries [J0, J1): I_up reconstructed at the face centre
// from the upwind cell's stage-1 intensity and limited gradient, own
// (u > 0, offset x_f - x_c) or the neighbour's (offset x_f - x_nbr'), so both
// sides of a face see the same value.  u as the fused step kernel forms it:
// float from the face slot and the pair's direction, double from the
// tabulated n_p . s; the antipode's u is -d - A w . n.
template <typename R, typename M, bool MOVING, int J0, int J1>
__device__ __forceinline__ void recon_chunk(const VLArgs<R> &a, int64_t c, int sub, int np,
                                            R (&acca)[M::PPT], R (&accb)[M::PPT]) {
  constexpr int PPT = M::PPT;
  const size_t plane = (size_t)a.n * a.RS, off = (size_t)c * a.RS;
  const R *Gx = a.G, *Gy = a.G + plane, *Gz = a.G + 2 * plane;
  R Ia[PPT], Ib[PPT], xa[PPT], xb[PPT], ya[PPT], yb[PPT], za[PPT], zb[PPT];
  load_entries<M, J0, J1>(a.Ih + off, sub, Ia, Ib, np);
  load_entries<M, J0, J1>(Gx + off, sub, xa, xb, np);
  load_entries<M, J0, J1>(Gy + off, sub, ya, yb, np);
  load_entries<M, J0, J1>(Gz + off, sub, za, zb, np);
  R nx[PPT], ny[PPT], nz[PPT];
#pragma unroll
  for (int j = J0; j < J1; ++j) {
    if constexpr (sizeof(R) == 4)
      load_dir(a.dir, (M::FULL || j < np) ? M::pair(j, sub) : 0, nx[j], ny[j], nz[j]);
    acca[j] = accb[j] = R(0);
  }
  const int64_t k0 = a.ptr[c], k1 = a.ptr[c + 1];
  for (int64_t k = k0; k < k1; ++k) {
    const Geo<R> g = load_geo(a.recon + 8 * k);
    const size_t no = (size_t)a.nbr[k] * a.RS;
    R va[PPT], vb[PPT], qxa[PPT], qxb[PPT], qya[PPT], qyb[PPT], qza[PPT], qzb[PPT];
    load_entries<M, J0, J1>(a.Ih + no, sub, va, vb, np);
    load_entries<M, J0, J1>(Gx + no, sub, qxa, qxb, np);
    load_entries<M, J0, J1>(Gy + no, sub, qya, qyb, np);
    load_entries<M, J0, J1>(Gz + no, sub, qza, qzb, np);
    SlotF sl{0, 0, 0, 0};
    R w = R(0);
    if constexpr (sizeof(R) == 4) {
      sl = load_slot<float>(a.slotf + k);
      if (MOVING) w = sl.w;
    } else if (MOVING) {
      w = R(a.wface[k]);
    }
#pragma unroll
    for (int j = J0; j < J1; ++j) {
      R d;
      if constexpr (sizeof(R) == 4)
        d = slot_dot(nx[j], ny[j], nz[j], sl);
      else
        d = (M::FULL || j < np) ? R(a.uface[(size_t)k * a.H + M::pair(j, sub)]) : R(0);
      if (MOVING) {
        const R ua = d - w, ub = -d - w;
        const R oa = Ia[j] + (xa[j] * g.ox + ya[j] * g.oy + za[j] * g.oz);
        const R ob = Ib[j] + (xb[j] * g.ox + yb[j] * g.oy + zb[j] * g.oz);
        const R ia = va[j] + (qxa[j] * g.rx + qya[j] * g.ry + qza[j] * g.rz);
        const R ib = vb[j] + (qxb[j] * g.rx + qyb[j] * g.ry + qzb[j] * g.rz);
        acca[j] = fma(ua, positive(ua) ? oa : ia, acca[j]);
        accb[j] = fma(ub, positive(ub) ? ob : ib, accb[j]);
      } else {
        // u_a = d, u_b = -d: one angle of the pair leaves through the face
        // (own value), the other enters (the neighbour's value)
        const bool out = positive(d);
        const R oI = out ? Ia[j] : Ib[j], oX = out ? xa[j] : xb[j], oY = out ? ya[j] : yb[j],
                oZ = out ? za[j] : zb[j];
        const R nI = out ? vb[j] : va[j], nX = out ? qxb[j] : qxa[j],
                nY = out ? qyb[j] : qya[j], nZ = out ? qzb[j] : qza[j];
        const R vo = oI + (oX * g.ox + oY * g.oy + oZ * g.oz);
        const R vn = nI + (nX * g.rx + nY * g.ry + nZ * g.rz);
        acca[j] = fma(d, out ? vo : vn, acca[j]);
        accb[j] = fma(-d, out ? vn : vo, accb[j]);
      }
    }
  }
}

template <typename R, typename M, bool MOVING, int CJ, int J0>
__device__ __forceinline__ void recon_chunks(const VLArgs<R> &a, int64_t c, int sub, int np,
                                             R (&acca)[M::PPT], R (&accb)[M::PPT]) {
  if constexpr (J0 < M::PPT) {
    constexpr int J1 = chunk_end<M, CJ, J0>();
    recon_chunk<R, M, MOVING, J0, J1>(a, c, sub, np, acca, accb);
    recon_chunks<R, M, MOVING, CJ, J1>(a, c, sub, np, acca, accb);
  }
}

// I* = I^n - dt/V_c sum_f u I_up.
template <typename R, typename M, bool MOVING, int CJ>
__global__ void __launch_bounds__(NT, 2) recon_transport_tile(const VLArgs<R> a) {
  constexpr int PPT = M::PPT;
  const int lc = threadIdx.x / KT, sub = threadIdx.x % KT;
  const int64_t c = (int64_t)blockIdx.x * CPB + lc;
  if (c >= a.n) return;  // no barrier below
  const int np = M::count(a.H, sub);
  R acca[PPT], accb[PPT];
  recon_chunks<R, M, MOVING, CJ, 0>(a, c, sub, np, acca, accb);
  R Ia[PPT], Ib[PPT];
  M::load(a.I + (size_t)c * a.RS, sub, Ia, Ib, np);
  const R dtv = a.dt * a.inv_vol[c];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    Ia[j] = fma(-dtv, acca[j], Ia[j]);
    Ib[j] = fma(-dtv, accb[j], Ib[j]);
  }
  M::store(a.Istar + (size_t)c * a.RS, sub, Ia, Ib, np);
}

// ---------------------------------------------------------------- quad rows
// Float rows in the quad layout.  A thread's angles come as float2 units:
// (p, p+1) and (p+H, p+1+H) of each of its quads, (q, q+H) of its tail pair,
// so that the arithmetic runs on packed FP32 pairs.  The block's face records
// (x_f - x_c, w_f | x_f - x_nbr', nbr) and, for the transport, its slots are
// copied into shared memory first.  The units of one pass: quads [Q0, Q1)
// and the tail pair if T; a pass walks the cell's faces.

__device__ __forceinline__ float2 pmax0(float2 v) {
  return make_float2(fmaxf(v.x, 0.0f), fmaxf(v.y, 0.0f));
}
__device__ __forceinline__ float2 pmin0(float2 v) {
  return make_float2(fminf(v.x, 0.0f), fminf(v.y, 0.0f));
}
__device__ __forceinline__ float2 pmin(float2 a, float2 b) {
  return make_float2(fminf(a.x, b.x), fminf(a.y, b.y));
}
__device__ __forceinline__ float2 pmax(float2 a, float2 b) {
  return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y));
}
__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }
// i + (x o_x + y o_y + z o_z), the face value of a unit, in the oracle's order
__device__ __forceinline__ float2 face_value(float2 i, float2 x, float2 y, float2 z, float2 ox,
                                             float2 oy, float2 oz) {
  return padd(i, pfma(z, oz, pfma(y, oy, pmul(x, ox))));
}

template <int Q0, int Q1, bool T> constexpr int kUnits = 2 * (Q1 - Q0) + (T ? 1 : 0);

template <int Q4, int Q0, int Q1, bool T>
__device__ __forceinline__ void load_units(const float *__restrict__ row, int sub,
                                           float2 (&x)[kUnits<Q0, Q1, T>]) {
  const float4 *q = reinterpret_cast<const float4 *>(row) + sub;
#pragma unroll
  for (int i = Q0; i < Q1; ++i) {
    const float4 t = q[KT * i];
    x[2 * (i - Q0)] = make_float2(t.x, t.y);
    x[2 * (i - Q0) + 1] = make_float2(t.z, t.w);
  }
  if (T) x[kUnits<Q0, Q1, T> - 1] = reinterpret_cast<const float2 *>(row)[16 * Q4 + sub];
}
template <int Q4, int Q0, int Q1, bool T>
__device__ __forceinline__ void store_units(float *__restrict__ row, int sub,
                                            const float2 (&x)[kUnits<Q0, Q1, T>]) {
  float4 *q = reinterpret_cast<float4 *>(row) + sub;
#pragma unroll
  for (int i = Q0; i < Q1; ++i)
    q[KT * i] = make_float4(x[2 * (i - Q0)].x, x[2 * (i - Q0)].y, x[2 * (i - Q0) + 1].x,
                            x[2 * (i - Q0) + 1].y);
  if (T) reinterpret_cast<float2 *>(row)[16 * Q4 + sub] = x[kUnits<Q0, Q1, T> - 1];
}

// All threads: copies of the block's face records (and slots) into shared
// memory; returns the block's first slot.
template <bool SLOTS>
__device__ __forceinline__ int64_t stage_faces(const VLArgs<float> &a, float4 *geo, SlotF *slot) {
  const int64_t c0 = (int64_t)blockIdx.x * CPB;
  const int64_t c1 = c0 + CPB < a.n ? c0 + CPB : a.n;
  const int64_t kb = a.ptr[c0];
  const int cnt = (int)(a.ptr[c1] - kb);
  const float4 *g = reinterpret_cast<const float4 *>(a.recon) + 2 * kb;
  for (int i = threadIdx.x; i < 2 * cnt; i += NT) cp_async16(geo + i, g + i);
  if (SLOTS)
    for (int i = threadIdx.x; i < cnt; i += NT) cp_async16(slot + i, a.slotf + kb + i);
  cp_async_wait_all();
  __syncthreads();
  return kb;
}

// The limited gradient of one pass's units (see gradient_chunk).
template <int Q4, int Q0, int Q1, bool T>
__device__ __forceinline__ void gradient_units(const VLArgs<float> &a, const float4 *geo, int k0,
                                               int k1, int64_t c, int sub, bool live) {
  constexpr int U = kUnits<Q0, Q1, T>;
  const size_t off = (size_t)c * a.RS;
  float2 I[U], BX[U], BY[U], BZ[U], LO[U], HI[U];
  load_units<Q4, Q0, Q1, T>(a.Ih + off, sub, I);
  const float2 z2 = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    BX[u] = BY[u] = BZ[u] = z2;
    LO[u] = HI[u] = I[u];
  }
  for (int k = k0; k < k1; ++k) {
    const float4 g0 = geo[2 * k], g1 = geo[2 * k + 1];
    const float2 WX = bc(g0.w * (g0.x - g1.x)), WY = bc(g0.w * (g0.y - g1.y)),
                 WZ = bc(g0.w * (g0.z - g1.z));
    float2 V[U];
    load_units<Q4, Q0, Q1, T>(a.Ih + (size_t)__float_as_int(g1.w) * a.RS, sub, V);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float2 D = psub(V[u], I[u]);
      BX[u] = pfma(WX, D, BX[u]);
      BY[u] = pfma(WY, D, BY[u]);
      BZ[u] = pfma(WZ, D, BZ[u]);
      LO[u] = pmin(LO[u], V[u]);
      HI[u] = pmax(HI[u], V[u]);
    }
  }
  const float *L = a.lsq + 8 * c;
  const float2 M00 = bc(L[0]), M01 = bc(L[1]), M02 = bc(L[2]), M11 = bc(L[3]), M12 = bc(L[4]),
               M22 = bc(L[5]);
  float2 GX[U], GY[U], GZ[U], XM[U], NM[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    GX[u] = pfma(M02, BZ[u], pfma(M01, BY[u], pmul(M00, BX[u])));
    GY[u] = pfma(M12, BZ[u], pfma(M11, BY[u], pmul(M01, BX[u])));
    GZ[u] = pfma(M22, BZ[u], pfma(M12, BY[u], pmul(M02, BX[u])));
    XM[u] = NM[u] = z2;
  }
  for (int k = k0; k < k1; ++k) {
    const float4 g0 = geo[2 * k];
    const float2 OX = bc(g0.x), OY = bc(g0.y), OZ = bc(g0.z);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float2 D = pfma(GZ[u], OZ, pfma(GY[u], OY, pmul(GX[u], OX)));
      XM[u] = pmax(XM[u], D);
      NM[u] = pmin(NM[u], D);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    float2 F = make_float2(1.0f, 1.0f);
    if (XM[u].x > 0.0f) F.x = fminf(F.x, (HI[u].x - I[u].x) / XM[u].x);
    if (NM[u].x < 0.0f) F.x = fminf(F.x, (LO[u].x - I[u].x) / NM[u].x);
    if (XM[u].y > 0.0f) F.y = fminf(F.y, (HI[u].y - I[u].y) / XM[u].y);
    if (NM[u].y < 0.0f) F.y = fminf(F.y, (LO[u].y - I[u].y) / NM[u].y);
    GX[u] = pmul(F, GX[u]);
    GY[u] = pmul(F, GY[u]);
    GZ[u] = pmul(F, GZ[u]);
  }
  if (live) {
    const size_t plane = (size_t)a.n * a.RS;
    store_units<Q4, Q0, Q1, T>(a.G + off, sub, GX);
    store_units<Q4, Q0, Q1, T>(a.G + plane + off, sub, GY);
    store_units<Q4, Q0, Q1, T>(a.G + 2 * plane + off, sub, GZ);
  }
}

// Passes over the units: the first takes the tail pair and up to (CP - 1) / 2
// quads, the others CP / 2 quads each (CP: pairs per pass).
template <int Q4, bool TAIL, int CP> struct QuadPasses {
  static constexpr int want = TAIL ? (CP - 1) / 2 : (CP / 2 > 0 ? CP / 2 : 1);
  static constexpr int first = want < Q4 ? want : Q4;
  __host__ __device__ static constexpr int end(int q0) {
    return q0 + (CP / 2 > 0 ? CP / 2 : 1) < Q4 ? q0 + (CP / 2 > 0 ? CP / 2 : 1) : Q4;
  }
};

template <int Q4, bool TAIL, int CP, int Q0, bool FIRST>
__device__ __forceinline__ void gradient_passes(const VLArgs<float> &a, const float4 *geo, int k0,
                                                int k1, int64_t c, int sub, bool live) {
  using P = QuadPasses<Q4, TAIL, CP>;
  if constexpr (FIRST) {
    gradient_units<Q4, 0, P::first, TAIL>(a, geo, k0, k1, c, sub, live);
    gradient_passes<Q4, TAIL, CP, P::first, false>(a, geo, k0, k1, c, sub, live);
  } else if constexpr (Q0 < Q4) {
    gradient_units<Q4, Q0, P::end(Q0), false>(a, geo, k0, k1, c, sub, live);
    gradient_passes<Q4, TAIL, CP, P::end(Q0), false>(a, geo, k0, k1, c, sub, live);
  }
}

template <int Q4, bool TAIL, int CP>
__global__ void __launch_bounds__(NT, 4) gradient_quad(const VLArgs<float> a) {
  extern __shared__ __align__(16) float4 vl_smem[];
  const int64_t kb = stage_faces<false>(a, vl_smem, nullptr);
  const int lc = threadIdx.x / KT, sub = threadIdx.x % KT;
  const int64_t cell = (int64_t)blockIdx.x * CPB + lc;
  const bool live = cell < a.n;
  const int64_t c = live ? cell : a.n - 1;  // dead lanes shadow the last cell
  gradient_passes<Q4, TAIL, CP, 0, true>(a, vl_smem, (int)(a.ptr[c] - kb), (int)(a.ptr[c + 1] - kb), c,
                                   sub, live);
}

// The reconstructed flux sums of one pass's units.  ACC holds the thread's
// accumulators: ACC[0] the tail pair's (sum u I_up, sum u' I_up) when the map
// has a tail, then per quad (sum u I_up) of (p, p+1) and (-sum u' I_up) of the
// antipodes.  The upwind choice as the step kernel makes it: max(u, 0) times
// the own face value plus min(u, 0) times the neighbour's, one of them zero.
template <int Q4, bool TAIL, bool MOVING, int Q0, int Q1, bool T>
__device__ __forceinline__ void transport_units(const VLArgs<float> &a, const float4 *geo,
                                                const SlotF *slot, int k0, int k1, int64_t c,
                                                int sub, float2 (&ACC)[2 * Q4 + (TAIL ? 1 : 0)]) {
  constexpr int U = kUnits<Q0, Q1, T>;
  constexpr int NQ = Q1 - Q0;
  constexpr int A0 = TAIL ? 1 : 0;  // accumulator of the first quad unit
  const size_t plane = (size_t)a.n * a.RS, off = (size_t)c * a.RS;
  const float *Gx = a.G, *Gy = a.G + plane, *Gz = a.G + 2 * plane;
  float2 I[U], X[U], Y[U], Z[U];
  load_units<Q4, Q0, Q1, T>(a.Ih + off, sub, I);
  load_units<Q4, Q0, Q1, T>(Gx + off, sub, X);
  load_units<Q4, Q0, Q1, T>(Gy + off, sub, Y);
  load_units<Q4, Q0, Q1, T>(Gz + off, sub, Z);
  float2 NX[NQ > 0 ? NQ : 1], NY[NQ > 0 ? NQ : 1], NZ[NQ > 0 ? NQ : 1];
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int p = 2 * (sub + KT * (Q0 + i));
    float x0, y0, z0, x1, y1, z1;
    load_dir(a.dir, p, x0, y0, z0);
    load_dir(a.dir, p + 1, x1, y1, z1);
    NX[i] = make_float2(x0, x1);
    NY[i] = make_float2(y0, y1);
    NZ[i] = make_float2(z0, z1);
  }
  float tx = 0.0f, ty = 0.0f, tz = 0.0f;
  if (T) load_dir(a.dir, 16 * Q4 + sub, tx, ty, tz);
  for (int k = k0; k < k1; ++k) {
    const float4 g0 = geo[2 * k], g1 = geo[2 * k + 1];
    const SlotF s = slot[k];
    const size_t no = (size_t)__float_as_int(g1.w) * a.RS;
    float2 V[U], QX[U], QY[U], QZ[U];
    load_units<Q4, Q0, Q1, T>(a.Ih + no, sub, V);
    load_units<Q4, Q0, Q1, T>(Gx + no, sub, QX);
    load_units<Q4, Q0, Q1, T>(Gy + no, sub, QY);
    load_units<Q4, Q0, Q1, T>(Gz + no, sub, QZ);
    const float2 OX = bc(g0.x), OY = bc(g0.y), OZ = bc(g0.z);
    const float2 RX = bc(g1.x), RY = bc(g1.y), RZ = bc(g1.z);
    const float2 SX = bc(s.sx), SY = bc(s.sy), SZ = bc(s.sz);
    const float w = MOVING ? s.w : 0.0f;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      const int ua = 2 * i, ub = 2 * i + 1;
      const float2 D = pfma(NX[i], SX, pfma(NY[i], SY, pmul(NZ[i], SZ)));
      const float2 Ua = MOVING ? psub(D, bc(w)) : D;  // u of (p, p+1)
      const float2 Eb = MOVING ? padd(D, bc(w)) : D;  // -u' of the antipodes
      const float2 voa = face_value(I[ua], X[ua], Y[ua], Z[ua], OX, OY, OZ);
      const float2 vob = face_value(I[ub], X[ub], Y[ub], Z[ub], OX, OY, OZ);
      const float2 vna = face_value(V[ua], QX[ua], QY[ua], QZ[ua], RX, RY, RZ);
      const float2 vnb = face_value(V[ub], QX[ub], QY[ub], QZ[ub], RX, RY, RZ);
      float2 &ca = ACC[A0 + 2 * (Q0 + i)], &cb = ACC[A0 + 2 * (Q0 + i) + 1];
      ca = pfma(pmax0(Ua), voa, pfma(pmin0(Ua), vna, ca));
      cb = pfma(pmin0(Eb), vob, pfma(pmax0(Eb), vnb, cb));
    }
    if (T) {
      const int ut = U - 1;
      const float d = fmaf(tx, s.sx, fmaf(ty, s.sy, tz * s.sz));
      const float2 Ut = make_float2(d - w, -d - w);
      const float2 vo = face_value(I[ut], X[ut], Y[ut], Z[ut], OX, OY, OZ);
      const float2 vn = face_value(V[ut], QX[ut], QY[ut], QZ[ut], RX, RY, RZ);
      ACC[0] = pfma(pmax0(Ut), vo, pfma(pmin0(Ut), vn, ACC[0]));
    }
  }
}

template <int Q4, bool TAIL, bool MOVING, int CP, int Q0, bool FIRST>
__device__ __forceinline__ void transport_passes(const VLArgs<float> &a, const float4 *geo,
                                                 const SlotF *slot, int k0, int k1, int64_t c,
                                                 int sub, float2 (&ACC)[2 * Q4 + (TAIL ? 1 : 0)]) {
  using P = QuadPasses<Q4, TAIL, CP>;
  if constexpr (FIRST) {
    transport_units<Q4, TAIL, MOVING, 0, P::first, TAIL>(a, geo, slot, k0, k1, c, sub, ACC);
    transport_passes<Q4, TAIL, MOVING, CP, P::first, false>(a, geo, slot, k0, k1, c, sub, ACC);
  } else if constexpr (Q0 < Q4) {
    transport_units<Q4, TAIL, MOVING, Q0, P::end(Q0), false>(a, geo, slot, k0, k1, c, sub, ACC);
    transport_passes<Q4, TAIL, MOVING, CP, P::end(Q0), false>(a, geo, slot, k0, k1, c, sub, ACC);
  }
}

// I* = I^n - dt/V_c sum_f u I_up over float rows in the quad layout (three
// blocks per SM measured faster than two at the register count the
// compiler picks unbounded).
template <int Q4, bool TAIL, bool MOVING, int CP>
__global__ void __launch_bounds__(NT, 3) recon_transport_quad(const VLArgs<float> a, int cap) {
  extern __shared__ __align__(16) float4 vl_smem[];
  SlotF *slot = reinterpret_cast<SlotF *>(vl_smem + 2 * cap);
  const int64_t kb = stage_faces<true>(a, vl_smem, slot);
  const int lc = threadIdx.x / KT, sub = threadIdx.x % KT;
  const int64_t cell = (int64_t)blockIdx.x * CPB + lc;
  const bool live = cell < a.n;
  const int64_t c = live ? cell : a.n - 1;  // dead lanes shadow the last cell
  constexpr int NA = 2 * Q4 + (TAIL ? 1 : 0);
  float2 ACC[NA];
#pragma unroll
  for (int u = 0; u < NA; ++u) ACC[u] = make_float2(0.0f, 0.0f);
  transport_passes<Q4, TAIL, MOVING, CP, 0, true>(a, vl_smem, slot, (int)(a.ptr[c] - kb),
                                            (int)(a.ptr[c + 1] - kb), c, sub, ACC);
  using M = QuadMap<Q4, TAIL>;
  float Ia[M::PPT], Ib[M::PPT];
  M::load(a.I + (size_t)c * a.RS, sub, Ia, Ib, M::PPT);
  const float dtv = a.dt * a.inv_vol[c];
  constexpr int A0 = TAIL ? 1 : 0;
#pragma unroll
  for (int i = 0; i < Q4; ++i) {
    // entries 2i, 2i+1 of the map are the pairs (p, p+1) of quad i
    Ia[2 * i] = fmaf(-dtv, ACC[A0 + 2 * i].x, Ia[2 * i]);
    Ia[2 * i + 1] = fmaf(-dtv, ACC[A0 + 2 * i].y, Ia[2 * i + 1]);
    Ib[2 * i] = fmaf(dtv, ACC[A0 + 2 * i + 1].x, Ib[2 * i]);
    Ib[2 * i + 1] = fmaf(dtv, ACC[A0 + 2 * i + 1].y, Ib[2 * i + 1]);
  }
  if (TAIL) {
    Ia[2 * Q4] = fmaf(-dtv, ACC[0].x, Ia[2 * Q4]);
    Ib[2 * Q4] = fmaf(-dtv, ACC[0].y, Ib[2 * Q4]);
  }
  if (live) M::store(a.Istar + (size_t)c * a.RS, sub, Ia, Ib, M::PPT);
}

template <int Q4, bool TAIL> cudaError_t vl_launch_quad(rt_state *s, const VLArgs<float> &a) {
  constexpr int CPG = 2, CPT = 3;  // pairs per pass: gradient, transport
  const unsigned blocks = (unsigned)((s->n_cells + CPB - 1) / CPB);
  const int cap = stage_cap(s->max_block_slots);
  gradient_quad<Q4, TAIL, CPG><<<blocks, NT, (size_t)cap * 32, s->stream>>>(a);
  if (s->moving)
    recon_transport_quad<Q4, TAIL, true, CPT><<<blocks, NT, (size_t)cap * 48, s->stream>>>(a, cap);
  else
    recon_transport_quad<Q4, TAIL, false, CPT><<<blocks, NT, (size_t)cap * 48, s->stream>>>(a, cap);
  s->launches += 2;
  return cudaGetLastError();
}

// Entries per chunk (what fits 128 registers without spills): float rows
// whole up to 5 pairs a thread (6 for the gradient), else 4 at a time;
// double rows 2 pairs at a time (each entry holds eight doubles of the cell
// and, in the transport, eight of the neighbour).
template <typename R, typename M, bool MOVING>
__host__ __device__ constexpr int transport_chunk() {
  return sizeof(R) == 8 ? 2 : (M::PPT <= 5 && !MOVING ? M::PPT : 4);
}
template <typename R, typename M> __host__ __device__ constexpr int gradient_chunk_size() {
  return sizeof(R) == 8 ? 2 : (M::PPT <= 6 ? M::PPT : 4);
}

template <typename R> VLArgs<R> vl_args(rt_state *s, double dt) {
  VLArgs<R> a{};
  a.n = s->n_cells;
  a.H = s->n_angles / 2;
  a.RS = s->row_stride;
  a.ptr = s->d_ptr;
  a.nbr = s->d_nbr;
  a.slotf = sizeof(R) == 4 ? reinterpret_cast<const SlotF *>(s->d_slot) : nullptr;
  a.uface = s->d_uface;
  a.wface = s->d_wface;
  a.recon = reinterpret_cast<const R *>(s->d_recon);
  a.lsq = reinterpret_cast<const R *>(s->d_lsq);
  a.dir = reinterpret_cast<const R *>(s->d_dir);
  a.inv_vol = reinterpret_cast<const R *>(s->d_inv_vol);
  a.I = reinterpret_cast<const R *>(s->d_I[s->cur]);
  a.Ih = reinterpret_cast<const R *>(s->d_Ihalf);
  a.G = reinterpret_cast<R *>(s->d_grad);
  a.Istar = reinterpret_cast<R *>(s->d_I[s->cur ^ 1]);
  a.dt = R(dt);
  return a;
}

template <typename R, typename M> cudaError_t vl_launch(rt_state *s, double dt) {
  const VLArgs<R> a = vl_args<R>(s, dt);
  const unsigned blocks = (unsigned)((s->n_cells + CPB - 1) / CPB);
  gradient_tile<R, M, gradient_chunk_size<R, M>()><<<blocks, NT, 0, s->stream>>>(a);
  if (s->moving)
    recon_transport_tile<R, M, true, transport_chunk<R, M, true>()>
        <<<blocks, NT, 0, s->stream>>>(a);
  else
    recon_transport_tile<R, M, false, transport_chunk<R, M, false>()>
        <<<blocks, NT, 0, s->stream>>>(a);
  s->launches += 2;
  return cudaGetLastError();
}

template <typename R, bool FULL> cudaError_t vl_pairs(rt_state *s, double dt) {
  switch ((s->n_angles / 2 + KT - 1) / KT) {
    case 1: return vl_launch<R, PairMap<R, 1, FULL>>(s, dt);
    case 2: return vl_launch<R, PairMap<R, 2, FULL>>(s, dt);
    case 3: return vl_launch<R, PairMap<R, 3, FULL>>(s, dt);
    case 4: return vl_launch<R, PairMap<R, 4, FULL>>(s, dt);
    case 5: return vl_launch<R, PairMap<R, 5, FULL>>(s, dt);
    case 6: return vl_launch<R, PairMap<R, 6, FULL>>(s, dt);
    case 7: return vl_launch<R, PairMap<R, 7, FULL>>(s, dt);
    case 8: return vl_launch<R, PairMap<R, 8, FULL>>(s, dt);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t vl_quads(rt_state *s, double dt) {
  const VLArgs<float> a = vl_args<float>(s, dt);
  switch (s->n_angles / 16) {
    case 2: return vl_launch_quad<1, false>(s, a);
    case 3: return vl_launch_quad<1, true>(s, a);
    case 4: return vl_launch_quad<2, false>(s, a);
    case 5: return vl_launch_quad<2, true>(s, a);
    case 6: return vl_launch_quad<3, false>(s, a);
    case 7: return vl_launch_quad<3, true>(s, a);
    case 8: return vl_launch_quad<4, false>(s, a);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R> cudaError_t vl_middle(rt_state *s, double dt) {
  if (sizeof(R) == 4 && s->quad_end > 0) return vl_quads(s, dt);  // rows in the quad layout
  return (s->n_angles / 2) % KT == 0 ? vl_pairs<R, true>(s, dt) : vl_pairs<R, false>(s, dt);
}

}  // namespace

cudaError_t launch_step_vl(rt_state *s, double dt) {
  // stage 1: first-order step over dt/2 into the half buffer, gas discarded
  const StepIO half{s->d_I[s->cur], s->d_Ihalf, false, false};
  cudaError_t e = launch_step_io(s, 0.5 * dt, half);
  if (e != cudaSuccess) return e;
  // stage 2: reconstructed fluxes of I^{n+1/2} applied to I^n (into the
  // output buffer), then the source over dt in place
  e = (s->precision == RT_FP32) ? vl_middle<float>(s, dt) : vl_middle<double>(s, dt);
  if (e != cudaSuccess) return e;
  const StepIO src{s->d_I[s->cur ^ 1], s->d_I[s->cur ^ 1], true, true};
  return launch_step_io(s, dt, src);
}

}  // namespace rt
