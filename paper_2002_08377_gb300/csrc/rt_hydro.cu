// Gas dynamics on the state's mesh, for radiation subcycled under a hydro
// step (Sec. 2: Eq. time evolution with the Euler fluxes; the Riemann-solver
// steps and the van Leer integrator of Sec. 2).
//
// The gas state is the one the radiation step exchanges energy and momentum
// with: rho (GasStatic::rho), m and the total energy density e (GasDyn).
// A hydro step
//   1. forms the primitives (rho, v, P) of every cell;
//   2. computes every face's flux once, from its first cell (left), its
//      second cell (right) and the face normal n_f (left to right): the HLLC
//      flux of Toro (Riemann Solvers and Numerical Methods for Fluid
//      Dynamics, Sec. 10.4) with Davis's wave-speed estimates, times the area
//      (hydro_flux_kernel, one thread per face);
//   3. updates every cell by the sum of its faces' fluxes in the cell's list
//      order, + for a face's first cell and - for its second
//      (hydro_update_kernel): each face's flux enters its two cells with
//      opposite signs, so mass, momentum and energy are conserved to
//      rounding, and the sum order is fixed (no atomics);
// once with the cell-centred states (order 1), or as the van Leer step
// (order 2): a half step over dt/2 with the cell-centred states, then the
// limited least-squares gradients of the half-step primitives
// (hydro_gradient_kernel: min sum A_f / |r|^2 (W_j - W_c - g . r)^2 over the
// face neighbours, r = x_j' - x_c, Barth-Jespersen limited to the range of the
// cell and its neighbours -- the reading of the gradient and limiter the
// radiation's reconstruction uses), and the full step over dt from the
// initial state with the fluxes of the primitives reconstructed at the face
// centroids.  Faces are static (the state's mesh).  Everything is double;
// this file is compiled without FMA contraction so that it rounds as the
// plain formulas do.  After the update the per-cell radiation coefficients
// (rho kappa, rho c_v, 1 / rho) follow the new density (opacities per unit
// mass are kept).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int kThreads = 256;

// primitive (rho, vx, vy, vz, P) of a conserved state
__device__ __forceinline__ void prim(double gamma, double rho, double mx, double my, double mz,
                                     double e, double *W) {
  W[0] = rho;
  W[1] = mx / rho;
  W[2] = my / rho;
  W[3] = mz / rho;
  W[4] = (gamma - 1.0) * (e - 0.5 * (mx * mx + my * my + mz * mz) / rho);
}

// HLLC flux per unit area through a face with unit normal n, left state WL
// on the side n points away from; returns false for a non-positive density
// or pressure.
__device__ bool hllc(double gamma, const double *WL, const double *WR, const double *n,
                     double *F) {
  const double *W[2] = {WL, WR};
  double u[2], a[2], E[2], Fk[2][5];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double *w = W[k];
    if (!(w[0] > 0.0) || !(w[4] > 0.0)) return false;
    u[k] = w[1] * n[0] + w[2] * n[1] + w[3] * n[2];
    a[k] = sqrt(gamma * w[4] / w[0]);
    E[k] = w[4] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
    Fk[k][0] = w[0] * u[k];
#pragma unroll
    for (int d = 0; d < 3; ++d) Fk[k][1 + d] = w[0] * w[1 + d] * u[k] + w[4] * n[d];
    Fk[k][4] = (E[k] + w[4]) * u[k];
  }
  // the slowest and fastest signal speeds (Davis) and the contact speed
  const double SL = fmin(u[0] - a[0], u[1] - a[1]);
  const double SR = fmax(u[0] + a[0], u[1] + a[1]);
  const double Ss = (WR[4] - WL[4] + WL[0] * u[0] * (SL - u[0]) - WR[0] * u[1] * (SR - u[1])) /
                    (WL[0] * (SL - u[0]) - WR[0] * (SR - u[1]));
  if (SL >= 0.0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = Fk[0][q];
  } else if (SR <= 0.0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = Fk[1][q];
  } else {
    // F*_K = F_K + S_K (U*_K - U_K) on the side of the contact that holds
    // the face, the star state carrying the tangential velocity unchanged
    const bool left = Ss >= 0.0;  // the side's values by selects (no indexed local arrays)
    const double S = left ? SL : SR, uk = left ? u[0] : u[1], Ek = left ? E[0] : E[1];
    double w[5], Fs[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      w[q] = left ? WL[q] : WR[q];
      Fs[q] = left ? Fk[0][q] : Fk[1][q];
    }
    const double f = w[0] * (S - uk) / (S - Ss);
    double Us[5], U[5];
    Us[0] = f;
#pragma unroll
    for (int d = 0; d < 3; ++d) Us[1 + d] = f * (w[1 + d] + (Ss - uk) * n[d]);
    Us[4] = f * (Ek / w[0] + (Ss - uk) * (Ss + w[4] / (w[0] * (S - uk))));
    U[0] = w[0];
#pragma unroll
    for (int d = 0; d < 3; ++d) U[1 + d] = w[0] * w[1 + d];
    U[4] = Ek;
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = Fs[q] + S * (Us[q] - U[q]);
  }
  return true;
}

// W[c][5] from (GasStatic::rho, GasDyn) or from U[c][5] = (rho, mx, my, mz, e);
// a non-positive density or pressure is latched in status
__global__ void prim_kernel(const GasStatic *__restrict__ gs, const GasDyn *__restrict__ gd,
                            const double *__restrict__ U, int64_t n, double gamma, double *W,
                            unsigned *status, unsigned long long *bad) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double *w = W + 5 * c;
  if (U)
    prim(gamma, U[5 * c], U[5 * c + 1], U[5 * c + 2], U[5 * c + 3], U[5 * c + 4], w);
  else
    prim(gamma, gs[c].rho, gd[c].mx, gd[c].my, gd[c].mz, gd[c].e, w);
  if (!(w[0] > 0.0) || !(w[4] > 0.0)) {
    atomicOr(status, ST_NONFINITE);
    atomicMin(bad, (unsigned long long)c);
  }
}

// area x HLLC flux of every face, from cell-centred or reconstructed states
__global__ void flux_kernel(const HydroFace *__restrict__ faces, int64_t nf,
                            const double *__restrict__ W, const double *__restrict__ grad,
                            double gamma, double *flux, unsigned *status,
                            unsigned long long *bad) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const HydroFace fc = faces[f];
  double WL[5], WR[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    WL[q] = W[5 * (int64_t)fc.i + q];
    WR[q] = W[5 * (int64_t)fc.j + q];
  }
  if (grad) {
    const double *gi = grad + 15 * (int64_t)fc.i, *gj = grad + 15 * (int64_t)fc.j;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      WL[q] += gi[q] * fc.oi[0] + gi[5 + q] * fc.oi[1] + gi[10 + q] * fc.oi[2];
      WR[q] += gj[q] * fc.oj[0] + gj[5 + q] * fc.oj[1] + gj[10 + q] * fc.oj[2];
    }
  }
  double F[5];
  double *out = flux + 5 * f;
  if (!hllc(gamma, WL, WR, fc.n, F)) {
    atomicOr(status, ST_NONFINITE);
    atomicMin(bad, (unsigned long long)fc.i);
#pragma unroll
    for (int q = 0; q < 5; ++q) out[q] = 0.0;
    return;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) out[q] = fc.area * F[q];
}

// U_out = U_in - h / V sum over the cell's slots in list order of
// sign x face flux.  U_in / U_out: (rho, m, e) either as (GasStatic::rho,
// GasDyn) or as U[c][5]; rho_out may be a plain array.
__global__ void update_kernel(const int64_t *__restrict__ ptr, const HydroSlot *__restrict__ slot,
                              const double *__restrict__ flux, const double *__restrict__ vol,
                              int64_t n, double h, const GasStatic *__restrict__ gs_in,
                              const GasDyn *__restrict__ gd_in, double *U_out,
                              double *rho_out, GasDyn *gd_out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t k = ptr[c]; k < ptr[c + 1]; ++k) {
    const HydroSlot sl = slot[k];
    const double *F = flux + 5 * (int64_t)sl.face;
#pragma unroll
    for (int q = 0; q < 5; ++q) s[q] += sl.sign * F[q];
  }
  const double hv = h / vol[c];
  const GasDyn d = gd_in[c];
  const double r = gs_in[c].rho - hv * s[0];
  const double mx = d.mx - hv * s[1], my = d.my - hv * s[2], mz = d.mz - hv * s[3];
  const double e = d.e - hv * s[4];
  if (U_out) {
    double *u = U_out + 5 * c;
    u[0] = r;
    u[1] = mx;
    u[2] = my;
    u[3] = mz;
    u[4] = e;
  } else {
    rho_out[c] = r;
    gd_out[c] = GasDyn{e, mx, my, mz};
  }
}

// The static part of the least-squares gradients, once per state (the faces
// do not move): per slot the weight A_f / |r|^2 times r = x_f - x_c - (x_f
// - x_j'), and per cell the cofactors C and the determinant of the normal
// matrix M = sum over the slots in list order of (A_f / |r|^2) r r^T, each
// rounded as the per-step formula would round it.
__global__ void lsq_setup_kernel(const int64_t *__restrict__ ptr, HydroSlot *slot, int64_t n,
                                 double *lsq) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int64_t k = ptr[c]; k < ptr[c + 1]; ++k) {
    HydroSlot &sl = slot[k];
    const double r[3] = {sl.own[0] - sl.nbr[0], sl.own[1] - sl.nbr[1], sl.own[2] - sl.nbr[2]};
    const double w = sl.area / (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const double wr[3] = {w * r[0], w * r[1], w * r[2]};
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      sl.wr[x] = wr[x];
#pragma unroll
      for (int y = 0; y < 3; ++y) M[x][y] += wr[x] * r[y];
    }
  }
  double *C = lsq + 10 * c;  // C[3 x + y], then the determinant
  C[0] = M[1][1] * M[2][2] - M[1][2] * M[2][1];
  C[1] = M[0][2] * M[2][1] - M[0][1] * M[2][2];
  C[2] = M[0][1] * M[1][2] - M[0][2] * M[1][1];
  C[3] = M[1][2] * M[2][0] - M[1][0] * M[2][2];
  C[4] = M[0][0] * M[2][2] - M[0][2] * M[2][0];
  C[5] = M[0][2] * M[1][0] - M[0][0] * M[1][2];
  C[6] = M[1][0] * M[2][1] - M[1][1] * M[2][0];
  C[7] = M[0][1] * M[2][0] - M[0][0] * M[2][1];
  C[8] = M[0][0] * M[1][1] - M[0][1] * M[1][0];
  C[9] = M[0][0] * C[0] + M[0][1] * C[3] + M[0][2] * C[6];
}

// Limited least-squares gradients grad[c][3][5] of the primitives W[c][5]
// (x, y, z components of the five fields): g = M^-1 b with
// b = sum A_f / |r|^2 r (W_j - W_c) over the cell's slots in list order (the
// static weights and the inverse by cofactors from lsq_setup_kernel).  Two
// passes over the cell's slots serve all five fields: the first forms the
// right-hand sides and the neighbour range, the second the extreme face
// increments g . (x_f - x_c).  The Barth-Jespersen factor min_f (hi - v) / dv
// (dv > 0) or (lo - v) / dv (dv < 0) is taken as one division by the largest
// positive and one by the most negative increment: the numerators have fixed
// signs and correctly rounded division is monotone in the divisor, so the
// minimum is the same number.
__global__ void __launch_bounds__(kThreads, 2)
    gradient_kernel(const int64_t *__restrict__ ptr, const int32_t *__restrict__ nbr,
                    const HydroSlot *__restrict__ slot, const double *__restrict__ lsq,
                    const double *__restrict__ W, int64_t n, double *grad) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int64_t k0 = ptr[c], k1 = ptr[c + 1];
  const double *Wc = W + 5 * c;
  double v[5], lo[5], hi[5], b[5][3];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    v[q] = Wc[q];
    lo[q] = v[q];
    hi[q] = v[q];
    b[q][0] = b[q][1] = b[q][2] = 0.0;
  }
  for (int64_t k = k0; k < k1; ++k) {
    const double wr[3] = {slot[k].wr[0], slot[k].wr[1], slot[k].wr[2]};
    const double *Wj = W + 5 * (int64_t)nbr[k];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const double vj = Wj[q];
#pragma unroll
      for (int x = 0; x < 3; ++x) b[q][x] += wr[x] * (vj - v[q]);
      lo[q] = fmin(lo[q], vj);
      hi[q] = fmax(hi[q], vj);
    }
  }
  const double *C = lsq + 10 * c;
  const double det = C[9];
  double g[5][3], dmax[5], dmin[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
#pragma unroll
    for (int x = 0; x < 3; ++x)
      g[q][x] = (C[3 * x] * b[q][0] + C[3 * x + 1] * b[q][1] + C[3 * x + 2] * b[q][2]) / det;
    dmax[q] = 0.0;
    dmin[q] = 0.0;
  }
  for (int64_t k = k0; k < k1; ++k) {
    const double o0 = slot[k].own[0], o1 = slot[k].own[1], o2 = slot[k].own[2];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const double dv = g[q][0] * o0 + g[q][1] * o1 + g[q][2] * o2;
      dmax[q] = fmax(dmax[q], dv);
      dmin[q] = fmin(dmin[q], dv);
    }
  }
  double *out = grad + 15 * c;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    // Barth-Jespersen: the largest factor keeping every face value in [lo, hi]
    double alpha = 1.0;
    if (dmax[q] > 0.0) alpha = fmin(alpha, (hi[q] - v[q]) / dmax[q]);
    if (dmin[q] < 0.0) alpha = fmin(alpha, (lo[q] - v[q]) / dmin[q]);
#pragma unroll
    for (int x = 0; x < 3; ++x) out[5 * x + q] = g[q][x] * alpha;
  }
}

// The radiation's per-cell coefficients from the new density: rho kappa
// with the opacities per unit mass, rho c_v, 1 / rho and their float copies.
__global__ void refresh_kernel(const double *__restrict__ rho, const double *__restrict__ kmass,
                               int64_t n, double cv, GasStatic *gs) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double r = rho[c];
  GasStatic g;
  g.rho = r;
  g.rkP = r * kmass[3 * c];
  g.rkJ = r * kmass[3 * c + 1];
  g.rkS = r * kmass[3 * c + 2];
  g.inv_rho = 1.0 / r;
  g.rcv = r * cv;
  g.frkP = (float)g.rkP;
  g.frkJ = (float)g.rkJ;
  g.frkS = (float)g.rkS;
  g.frcv = (float)g.rcv;
  gs[c] = g;
}

// cfl V^(1/3) / (|v| + sound speed), minimum over cells (positive doubles
// order as their bit patterns)
__global__ void dt_kernel(const GasStatic *__restrict__ gs, const GasDyn *__restrict__ gd,
                          const double *__restrict__ vol, int64_t n, double gamma, double cfl,
                          unsigned long long *best) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double W[5];
  prim(gamma, gs[c].rho, gd[c].mx, gd[c].my, gd[c].mz, gd[c].e, W);
  const double v = sqrt(W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
  const double a = sqrt(gamma * W[4] / W[0]);
  const double t = cfl * (cbrt(vol[c]) / (v + a));
  if (t > 0.0) atomicMin(best, (unsigned long long)__double_as_longlong(t));
}

unsigned grid(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

int hydro_setup(rt_state *s, const rt_mesh_desc *m) {
  const int64_t N = s->n_cells, Nf = m->n_faces;
  std::vector<int64_t> slot_of(N);
  for (int64_t ic = 0; ic < N; ++ic) slot_of[s->cell_of[ic]] = ic;
  std::vector<HydroFace> faces(Nf);
  for (int64_t f = 0; f < Nf; ++f) {
    HydroFace &h = faces[f];
    h.i = (int32_t)slot_of[m->face_cells[2 * f]];
    h.j = (int32_t)slot_of[m->face_cells[2 * f + 1]];
    h.area = m->face_area[f];
    for (int d = 0; d < 3; ++d) {
      h.n[d] = m->face_normal[3 * f + d];
      h.oi[d] = m->face_offset[6 * f + d];
      h.oj[d] = m->face_offset[6 * f + 3 + d];
    }
  }
  std::vector<HydroSlot> slots(s->nnz);
  int64_t o = 0;
  for (int64_t ic = 0; ic < N; ++ic) {
    const int64_t c = s->cell_of[ic];
    for (int64_t k = m->cell_face_ptr[c]; k < m->cell_face_ptr[c + 1]; ++k, ++o) {
      const int32_t e = m->cell_face_idx[k];
      const int64_t f = e >= 0 ? e : -(int64_t)e - 1;
      const bool first = e >= 0;
      HydroSlot &h = slots[o];
      for (int d = 0; d < 3; ++d) {
        h.own[d] = m->face_offset[6 * f + (first ? 0 : 3) + d];
        h.nbr[d] = m->face_offset[6 * f + (first ? 3 : 0) + d];
      }
      h.area = m->face_area[f];
      h.sign = first ? 1.0 : -1.0;
      h.face = f;
    }
  }
  cudaError_t e;
  auto up = [&](void **dst, const void *src, size_t bytes) {
    e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) s->device_bytes += bytes;
    return e == cudaSuccess;
  };
  if (!up((void **)&s->d_hface, faces.data(), sizeof(HydroFace) * Nf) ||
      !up((void **)&s->d_hslot, slots.data(), sizeof(HydroSlot) * s->nnz))
    return e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;
  e = cudaMalloc((void **)&s->d_hlsq, sizeof(double) * 10 * (size_t)N);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;
  s->device_bytes += sizeof(double) * 10 * (size_t)N;
  lsq_setup_kernel<<<grid(N), kThreads, 0, s->stream>>>(s->d_ptr, s->d_hslot, N, s->d_hlsq);
  s->launches++;
  e = cudaGetLastError();
  if (e != cudaSuccess) return RT_ERR_CUDA;
  const size_t work = sizeof(double) * ((size_t)N * (5 + 15 + 5 + 1 + 3) + (size_t)Nf * 5);
  e = cudaMalloc((void **)&s->d_hwork, work);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;
  s->device_bytes += work;
  return RT_OK;
}

// The work area: W[N][5], grad[N][15], U half step [N][5], rho [N],
// opacities per unit mass [N][3], face fluxes [Nf][5].
static double *work_W(rt_state *s) { return s->d_hwork; }
static double *work_grad(rt_state *s) { return s->d_hwork + 5 * s->n_cells; }
static double *work_U(rt_state *s) { return s->d_hwork + 20 * s->n_cells; }
static double *work_rho(rt_state *s) { return s->d_hwork + 25 * s->n_cells; }
double *hydro_kmass(rt_state *s) { return s->d_hwork + 26 * s->n_cells; }
static double *work_flux(rt_state *s) { return s->d_hwork + 29 * s->n_cells; }

cudaError_t launch_hydro_step(rt_state *s, double dt, int order) {
  const int64_t N = s->n_cells, Nf = s->n_faces;
  const double g = s->params.gamma_gas;
  double *W = work_W(s), *grad = work_grad(s), *U = work_U(s), *rho = work_rho(s);
  double *flux = work_flux(s);
  prim_kernel<<<grid(N), kThreads, 0, s->stream>>>(s->d_gs, s->d_gd, nullptr, N, g, W, s->d_status,
                                                   s->d_bad);
  flux_kernel<<<grid(Nf), kThreads, 0, s->stream>>>(s->d_hface, Nf, W, nullptr, g, flux,
                                                    s->d_status, s->d_bad);
  s->launches += 2;
  if (order == 1) {
    update_kernel<<<grid(N), kThreads, 0, s->stream>>>(s->d_ptr, s->d_hslot, flux, s->d_volume, N,
                                                       dt, s->d_gs, s->d_gd, nullptr, rho, s->d_gd);
    s->launches++;
  } else {
    // half step into U, gradients of its primitives, full step from the start
    update_kernel<<<grid(N), kThreads, 0, s->stream>>>(s->d_ptr, s->d_hslot, flux, s->d_volume, N,
                                                       0.5 * dt, s->d_gs, s->d_gd, U, nullptr,
                                                       nullptr);
    prim_kernel<<<grid(N), kThreads, 0, s->stream>>>(nullptr, nullptr, U, N, g, W, s->d_status,
                                                     s->d_bad);
    gradient_kernel<<<grid(N), kThreads, 0, s->stream>>>(s->d_ptr, s->d_nbr, s->d_hslot,
                                                         s->d_hlsq, W, N, grad);
    flux_kernel<<<grid(Nf), kThreads, 0, s->stream>>>(s->d_hface, Nf, W, grad, g, flux,
                                                      s->d_status, s->d_bad);
    update_kernel<<<grid(N), kThreads, 0, s->stream>>>(s->d_ptr, s->d_hslot, flux, s->d_volume, N,
                                                       dt, s->d_gs, s->d_gd, nullptr, rho, s->d_gd);
    s->launches += 5;
  }
  // the radiation's per-cell coefficients follow the new density, and the
  // new primitives are checked
  refresh_kernel<<<grid(N), kThreads, 0, s->stream>>>(rho, hydro_kmass(s), N,
                                                      s->params.r_gas / (g - 1.0), s->d_gs);
  prim_kernel<<<grid(N), kThreads, 0, s->stream>>>(s->d_gs, s->d_gd, nullptr, N, g, W, s->d_status,
                                                   s->d_bad);
  s->launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_cellv(s);
  return e;
}

cudaError_t launch_hydro_dt(rt_state *s, double cfl, double *dt) {
  unsigned long long *best = reinterpret_cast<unsigned long long *>(s->d_out16);
  const unsigned long long init = 0x7ff0000000000000ull;  // +inf
  cudaError_t e = cudaMemcpyAsync(best, &init, sizeof init, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return e;
  dt_kernel<<<grid(s->n_cells), kThreads, 0, s->stream>>>(s->d_gs, s->d_gd, s->d_volume,
                                                          s->n_cells, s->params.gamma_gas, cfl,
                                                          best);
  s->launches++;
  unsigned long long bits = 0;
  e = cudaMemcpyAsync(&bits, best, sizeof bits, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) std::memcpy(dt, &bits, sizeof bits);
  return e;
}

namespace {
__global__ void density_out_kernel(const GasStatic *__restrict__ gs,
                                   const int64_t *__restrict__ cell_of, int64_t n, double *rho) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rho[cell_of[i]] = gs[i].rho;
}
}  // namespace

cudaError_t launch_density_out(rt_state *s, double *rho) {
  density_out_kernel<<<grid(s->n_cells), kThreads, 0, s->stream>>>(s->d_gs, s->d_cell_of,
                                                                   s->n_cells, rho);
  s->launches++;
  return cudaGetLastError();
}

}  // namespace rt
