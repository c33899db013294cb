// Host side of the C ABI declared in include/rt.h: validation, locality
// ordering, directed face slots, device buffers and the call sequence.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <cuda.h>

#include "rt_internal.cuh"

namespace rt {
int64_t totals_scratch_len(int64_t n_cells);

void *driver_fn(const char *name) {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion(name, &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return fn;
}

unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent cur = reinterpret_cast<GetCurrent>(driver_fn("cuCtxGetCurrent"));
  static GetId id = reinterpret_cast<GetId>(driver_fn("cuCtxGetId"));
  CUcontext ctx = nullptr;
  unsigned long long v = 0;
  if (!cur || !id || cur(&ctx) != CUDA_SUCCESS || !ctx || id(ctx, &v) != CUDA_SUCCESS) return 0;
  return v;
}
}  // namespace rt

namespace {

int fail(rt_state *s, int code, const std::string &msg) {
  if (s) s->err = msg;
  return code;
}

int cuda_fail(rt_state *s, cudaError_t e, const char *what) {
  return fail(s, e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define RT_CUDA(s, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
  } while (0)

template <typename T> cudaError_t dalloc(rt_state *s, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e == cudaSuccess) s->device_bytes += count * sizeof(T);
  return e;
}

cudaError_t dalloc_bytes(rt_state *s, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) s->device_bytes += bytes;
  return e;
}

// Interleave the bits of a 21-bit integer with two zero bits.
uint64_t spread3(uint64_t v) {
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffull;
  v = (v | v << 16) & 0x1f0000ff0000ffull;
  v = (v | v << 8) & 0x100f00f00f00f00full;
  v = (v | v << 4) & 0x10c30c30c30c30c3ull;
  v = (v | v << 2) & 0x1249249249249249ull;
  return v;
}

// Locality order: sort cells along a Morton curve of their centroids.
std::vector<int64_t> morton_order(int64_t n, const double *cen) {
  std::vector<int64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  if (!cen || n < 2) return order;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t c = 0; c < n; ++c)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], cen[3 * c + d]);
      hi[d] = std::max(hi[d], cen[3 * c + d]);
    }
  std::vector<uint64_t> key(n);
  for (int64_t c = 0; c < n; ++c) {
    uint64_t k = 0;
    for (int d = 0; d < 3; ++d) {
      double span = hi[d] - lo[d];
      double t = span > 0 ? (cen[3 * c + d] - lo[d]) / span : 0.0;
      uint64_t q = (uint64_t)std::min(2097151.0, std::max(0.0, t * 2097151.0));
      k |= spread3(q) << d;
    }
    key[c] = k;
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  return order;
}

template <typename R> void fill_geometry(rt_state *s, const rt_mesh_desc *m,
                                         const std::vector<int64_t> &slot_of,
                                         std::vector<int64_t> &ptr, std::vector<int32_t> &nbr,
                                         std::vector<typename rt::SlotOf<R>::type> &slot,
                                         std::vector<double> &wface, std::vector<R> &inv_vol) {
  const int64_t N = m->n_cells;
  ptr.assign(N + 1, 0);
  for (int64_t ic = 0; ic < N; ++ic) {
    int64_t c = s->cell_of[ic];
    ptr[ic + 1] = ptr[ic] + (m->cell_face_ptr[c + 1] - m->cell_face_ptr[c]);
  }
  nbr.resize(ptr[N]);
  slot.resize(ptr[N]);
  wface.assign(sizeof(R) == 8 ? ptr[N] : 0, 0.0);
  inv_vol.resize(N);
  // float slots of a double state (the positivity screen's temporary copy)
  // are scaled by the power of two screen_scale so that they fit float at
  // any unit scale; a float state's own slots are unscaled (screen_scale 1)
  const double cbar = s->params.cbar * (sizeof(R) == 4 ? s->screen_scale : 1.0);
  const double wsc = sizeof(R) == 4 ? s->screen_scale : 1.0;
  for (int64_t ic = 0; ic < N; ++ic) {
    const int64_t c = s->cell_of[ic];
    inv_vol[ic] = (R)(1.0 / m->cell_volume[c]);
    int64_t o = ptr[ic];
    for (int64_t k = m->cell_face_ptr[c]; k < m->cell_face_ptr[c + 1]; ++k, ++o) {
      const int32_t e = m->cell_face_idx[k];
      const int64_t f = e >= 0 ? e : -(int64_t)e - 1;
      const double sg = e >= 0 ? 1.0 : -1.0;
      const int64_t other = e >= 0 ? m->face_cells[2 * f + 1] : m->face_cells[2 * f];
      nbr[o] = (int32_t)slot_of[other];
      const double A = m->face_area[f];
      const double *n = m->face_normal + 3 * f;
      double wn = 0.0;
      if (m->face_w) {
        const double *w = m->face_w + 3 * f;
        wn = (w[0] * n[0] + w[1] * n[1]) + w[2] * n[2];
      }
      // both sides hold exact negatives of the same rounded numbers
      if (sizeof(R) == 4) {
        R sx = (R)(cbar * A * n[0]), sy = (R)(cbar * A * n[1]), sz = (R)(cbar * A * n[2]);
        R ww = (R)(wsc * A * wn);
        if (sg < 0) {
          sx = -sx;
          sy = -sy;
          sz = -sz;
          ww = -ww;
        }
        slot[o] = {sx, sy, sz, ww};
      } else {
        slot[o] = {(R)(sg * n[0]), (R)(sg * n[1]), (R)(sg * n[2]), (R)(cbar * A)};
        wface[o] = A * (sg * wn);
      }
    }
  }
}

template <typename T> cudaError_t upload(rt_state *s, T **dst, const std::vector<T> &v) {
  cudaError_t e = dalloc(s, dst, v.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename R> int build_device_mesh(rt_state *s, const rt_mesh_desc *m,
                                            const std::vector<int64_t> &slot_of) {
  std::vector<int64_t> ptr;
  std::vector<int32_t> nbr;
  std::vector<typename rt::SlotOf<R>::type> slot;
  std::vector<double> wface;
  std::vector<R> inv_vol;
  fill_geometry<R>(s, m, slot_of, ptr, nbr, slot, wface, inv_vol);
  if (!wface.empty()) RT_CUDA(s, upload(s, &s->d_wface, wface));
  RT_CUDA(s, upload(s, &s->d_ptr, ptr));
  RT_CUDA(s, upload(s, &s->d_nbr, nbr));
  s->max_block_slots = 0;
  for (int64_t c0 = 0; c0 < m->n_cells; c0 += rt::CPB) {
    const int64_t c1 = std::min<int64_t>(m->n_cells, c0 + rt::CPB);
    s->max_block_slots = std::max(s->max_block_slots, ptr[c1] - ptr[c0]);
  }
  typename rt::SlotOf<R>::type *ds = nullptr;
  RT_CUDA(s, upload(s, &ds, slot));
  s->d_slot = ds;
  if constexpr (sizeof(R) == 4) {
    if (!s->moving) {
      // static float meshes: w = 0, so its word carries the neighbour index
      std::vector<rt::SlotF> snb(slot.size());
      for (size_t k = 0; k < slot.size(); ++k) {
        snb[k] = slot[k];
        std::memcpy(&snb[k].w, &nbr[k], sizeof(float));
      }
      RT_CUDA(s, upload(s, &s->d_slot_nb, snb));
    }
  }
  R *dv = nullptr;
  RT_CUDA(s, upload(s, &dv, inv_vol));
  s->d_inv_vol = dv;
  const int A = m->n_angles;
  std::vector<R> dir(4 * (size_t)A), wt(A);
  for (int a = 0; a < A; ++a) {
    for (int d = 0; d < 3; ++d) dir[4 * a + d] = (R)m->angle_dir[3 * a + d];
    dir[4 * a + 3] = 0;
  }
  for (int p = 0; p < A / 2; ++p) {  // (w_p, w_{p+A/2}) per pair
    wt[2 * p] = (R)m->angle_w[p];
    wt[2 * p + 1] = (R)m->angle_w[p + A / 2];
  }
  R *dd = nullptr, *dw = nullptr;
  RT_CUDA(s, upload(s, &dd, dir));
  RT_CUDA(s, upload(s, &dw, wt));
  s->d_dir = dd;
  s->d_wt = dw;
  return RT_OK;
}

// Linear-reconstruction geometry for the van Leer integrator, in the internal
// cell and slot order.  Per directed slot k of cell c (8 reals):
//   (x_f - x_c, w_f, x_f - x_nbr', nbr), w_f = A_f / |r_f|^2, r_f = x_nbr' - x_c,
// with nbr' the neighbour's image across f and nbr its internal index, kept
// as the bits of an int32 (float) or int64 (double) in the last real, so that
// one record carries everything a face of the reconstruction reads; per cell
// (8 reals) the inverse of
// M = sum_f w_f r_f r_f^T (symmetric: xx, xy, xz, yy, yz, zz, 0, 0), formed in
// double by cofactors.
template <typename R> int build_recon(rt_state *s, const rt_mesh_desc *m) {
  const int64_t N = m->n_cells;
  std::vector<R> rs(8 * (size_t)s->nnz), lsq(8 * (size_t)N, R(0));
  std::vector<int32_t> nbr((size_t)s->nnz);
  RT_CUDA(s, cudaMemcpy(nbr.data(), s->d_nbr, nbr.size() * sizeof(int32_t),
                        cudaMemcpyDeviceToHost));
  int64_t o = 0;
  for (int64_t ic = 0; ic < N; ++ic) {
    const int64_t c = s->cell_of[ic];
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int64_t k = m->cell_face_ptr[c]; k < m->cell_face_ptr[c + 1]; ++k, ++o) {
      const int32_t e = m->cell_face_idx[k];
      const int64_t f = e >= 0 ? e : -(int64_t)e - 1;
      const double *off = m->face_offset + 6 * f;
      const double *own = e >= 0 ? off : off + 3, *oth = e >= 0 ? off + 3 : off;
      const double r[3] = {own[0] - oth[0], own[1] - oth[1], own[2] - oth[2]};
      const double w = m->face_area[f] / (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
      for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) M[x][y] += w * r[x] * r[y];
      R *q = rs.data() + 8 * o;
      q[0] = (R)own[0];
      q[1] = (R)own[1];
      q[2] = (R)own[2];
      q[3] = (R)w;
      q[4] = (R)oth[0];
      q[5] = (R)oth[1];
      q[6] = (R)oth[2];
      if constexpr (sizeof(R) == 4) {
        const int32_t nb = nbr[o];
        std::memcpy(&q[7], &nb, sizeof nb);
      } else {
        const int64_t nb = nbr[o];
        std::memcpy(&q[7], &nb, sizeof nb);
      }
    }
    const double C00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
    const double C01 = M[0][2] * M[2][1] - M[0][1] * M[2][2];
    const double C02 = M[0][1] * M[1][2] - M[0][2] * M[1][1];
    const double C11 = M[0][0] * M[2][2] - M[0][2] * M[2][0];
    const double C12 = M[0][2] * M[1][0] - M[0][0] * M[1][2];
    const double C22 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    const double det = M[0][0] * C00 + M[0][1] * (M[1][2] * M[2][0] - M[1][0] * M[2][2]) +
                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (!(std::fabs(det) > 0))
      return fail(s, RT_ERR_MESH, "a cell's face neighbours do not span 3-D (singular gradient)");
    R *q = lsq.data() + 8 * ic;
    q[0] = (R)(C00 / det);
    q[1] = (R)(C01 / det);
    q[2] = (R)(C02 / det);
    q[3] = (R)(C11 / det);
    q[4] = (R)(C12 / det);
    q[5] = (R)(C22 / det);
  }
  R *drs = nullptr, *dlsq = nullptr;
  RT_CUDA(s, upload(s, &drs, rs));
  RT_CUDA(s, upload(s, &dlsq, lsq));
  s->d_recon = drs;
  s->d_lsq = dlsq;
  return RT_OK;
}

int check_mesh(rt_state *s, const rt_mesh_desc *m) {
  const int64_t N = m->n_cells, Nf = m->n_faces;
  if (N < 1 || N > INT32_MAX || Nf < 0 || m->n_angles < 2 || (m->n_angles & 1))
    return fail(s, RT_ERR_ARG, "n_cells, n_faces or n_angles out of range (n_angles must be even)");
  if (m->n_angles > 128) return fail(s, RT_ERR_ARG, "at most 128 angles are supported");
  if (!m->cell_volume || !m->face_cells || !m->face_area || !m->face_normal ||
      !m->cell_face_ptr || !m->cell_face_idx || !m->angle_dir || !m->angle_w)
    return fail(s, RT_ERR_ARG, "required mesh array is NULL");
  const int A = m->n_angles, H = A / 2;
  double wsum = 0;
  for (int a = 0; a < A; ++a) {
    const double *d = m->angle_dir + 3 * a;
    if (!(std::fabs(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - 1.0) < 1e-12))
      return fail(s, RT_ERR_ARG, "angle directions must be unit vectors");
    if (!(m->angle_w[a] > 0)) return fail(s, RT_ERR_ARG, "angle weights must be positive");
    wsum += m->angle_w[a];
  }
  if (!(std::fabs(wsum - 1.0) < 1e-12)) return fail(s, RT_ERR_ARG, "angle weights must sum to 1");
  for (int a = 0; a < H; ++a)
    for (int d = 0; d < 3; ++d)
      if (m->angle_dir[3 * (a + H) + d] != -m->angle_dir[3 * a + d])
        return fail(s, RT_ERR_ARG, "angle set must satisfy dir[a + A/2] == -dir[a]");
  if (m->cell_face_ptr[0] != 0) return fail(s, RT_ERR_MESH, "cell_face_ptr[0] must be 0");
  for (int64_t c = 0; c < N; ++c)
    if (m->cell_face_ptr[c + 1] < m->cell_face_ptr[c])
      return fail(s, RT_ERR_MESH, "cell_face_ptr must be non-decreasing");
  const int64_t nnz = m->cell_face_ptr[N];
  if (nnz != 2 * Nf) return fail(s, RT_ERR_MESH, "CSR must list every face twice");
  for (int64_t f = 0; f < Nf; ++f) {
    int32_t i = m->face_cells[2 * f], j = m->face_cells[2 * f + 1];
    if (i < 0 || i >= N || j < 0 || j >= N) return fail(s, RT_ERR_MESH, "face cell index out of range");
    if (!(m->face_area[f] >= 0) || !std::isfinite(m->face_area[f]))
      return fail(s, RT_ERR_MESH, "face areas must be finite and non-negative");
  }
  std::vector<uint8_t> seen(2 * (size_t)Nf, 0);
  std::vector<double> closure(3 * (size_t)N, 0.0), asum(N, 0.0);
  for (int64_t c = 0; c < N; ++c) {
    if (!(m->cell_volume[c] > 0) || !std::isfinite(m->cell_volume[c]))
      return fail(s, RT_ERR_MESH, "cell volumes must be positive");
    for (int64_t k = m->cell_face_ptr[c]; k < m->cell_face_ptr[c + 1]; ++k) {
      int32_t e = m->cell_face_idx[k];
      int64_t f = e >= 0 ? e : -(int64_t)e - 1;
      if (f >= Nf) return fail(s, RT_ERR_MESH, "cell_face_idx out of range");
      int side = e >= 0 ? 0 : 1;
      if (m->face_cells[2 * f + side] != c)
        return fail(s, RT_ERR_MESH, "cell_face_idx entry does not match face_cells");
      if (seen[2 * f + side]++) return fail(s, RT_ERR_MESH, "face listed twice on one side");
      double sg = side ? -1.0 : 1.0, A = m->face_area[f];
      for (int d = 0; d < 3; ++d) closure[3 * c + d] += sg * A * m->face_normal[3 * f + d];
      asum[c] += A;
    }
  }
  for (int64_t c = 0; c < N; ++c) {
    double r = std::sqrt(closure[3 * c] * closure[3 * c] + closure[3 * c + 1] * closure[3 * c + 1] +
                         closure[3 * c + 2] * closure[3 * c + 2]);
    if (!(r <= 1e-9 * asum[c])) {
      char buf[128];
      snprintf(buf, sizeof buf, "cell %lld is not closed: |sum A n| = %.3g", (long long)c, r);
      return fail(s, RT_ERR_MESH, buf);
    }
  }
  return RT_OK;
}

// Float states store cbar A n_f, A w . n_f and 1/V in float and multiply
// them by float intensities: each stored magnitude and its reciprocal must
// be a normal float (|x| in [2^-125, 2^125], or exactly 0 for a face
// product), else the step would overflow or flush to zero without an error.
bool float_normal(double x) { return x >= 0x1p-125 && x <= 0x1p125; }

int check_float_range(rt_state *s, const rt_mesh_desc *m, double cbar) {
  char buf[200];
  for (int64_t f = 0; f < m->n_faces; ++f) {
    const double A = m->face_area[f], ca = cbar * A;
    double wn = 0.0;
    if (m->face_w) {
      const double *w = m->face_w + 3 * f;
      wn = std::fabs(A * std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
    }
    if ((ca != 0.0 && !float_normal(ca)) || (wn != 0.0 && !float_normal(wn))) {
      snprintf(buf, sizeof buf,
               "RT_FP32: face %lld has cbar A = %.3g or A |w| = %.3g outside float range "
               "(2^-125 .. 2^125); rescale the units or use RT_FP64",
               (long long)f, ca, wn);
      return fail(s, RT_ERR_ARG, buf);
    }
  }
  for (int64_t c = 0; c < m->n_cells; ++c)
    if (!float_normal(m->cell_volume[c])) {
      snprintf(buf, sizeof buf,
               "RT_FP32: cell %lld has volume %.3g outside float range (2^-125 .. 2^125); "
               "rescale the units or use RT_FP64",
               (long long)c, m->cell_volume[c]);
      return fail(s, RT_ERR_ARG, buf);
    }
  return RT_OK;
}

int sync_status(rt_state *s) {
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  if (s->io_out) RT_CUDA(s, cudaStreamSynchronize(s->io_out));  // rt_step_io's result copies
  unsigned st = 0;
  unsigned long long bad = 0;
  RT_CUDA(s, cudaMemcpy(&st, s->d_status, sizeof st, cudaMemcpyDeviceToHost));
  if (!st) return RT_OK;
  RT_CUDA(s, cudaMemcpy(&bad, s->d_bad, sizeof bad, cudaMemcpyDeviceToHost));
  long long cell = bad < (unsigned long long)s->n_cells ? (long long)s->cell_of[bad] : -1;
  char buf[160];
  if (st & rt::ST_NONFINITE) {
    snprintf(buf, sizeof buf, "non-finite intensity or temperature (first cell %lld)", cell);
    return fail(s, RT_ERR_NONFINITE, buf);
  }
  if (st & rt::ST_CFL) {
    snprintf(buf, sizeof buf,
             "dt exceeds the upwind positivity limit of a cell's current volume (first cell %lld)",
             cell);
    return fail(s, RT_ERR_CFL, buf);
  }
  snprintf(buf, sizeof buf, "temperature Newton iteration did not converge (first cell %lld)", cell);
  return fail(s, RT_ERR_NONCONV, buf);
}

}  // namespace

extern "C" {

int rt_create(const rt_mesh_desc *m_in, const rt_params *p, void *stream, rt_state **out) {
  if (!out) return RT_ERR_ARG;
  *out = nullptr;
  if (!m_in || !p) return RT_ERR_ARG;
  rt_state *s = new rt_state();
  // frequency groups: the kernels see n_groups copies of the base angle set,
  // group j's weights scaled by group_w[j], ordered first halves of all
  // groups then second halves (so angle k and k + A'/2 stay antipodes)
  rt_mesh_desc mx = *m_in;
  const rt_mesh_desc *m = &mx;
  std::vector<double> gdir, gwt;
  const int G = m_in->n_groups > 1 ? m_in->n_groups : 1;
  s->n_groups = G;
  if (G > 1) {
    const int Ab = m_in->n_angles, Hb = Ab / 2;
    double wsum = 0.0;
    bool ok = m_in->group_w && Ab >= 2 && !(Ab & 1) && (int64_t)G * Ab <= 128 && G <= 8 &&
              m_in->angle_dir && m_in->angle_w && p->integrator == RT_FIRST_ORDER && !p->boost &&
              !p->gcl && p->beta_P == 0.0 && p->beta_J == 0.0;
    for (int j = 0; ok && j < G; ++j) {
      ok = std::isfinite(m_in->group_w[j]) && m_in->group_w[j] > 0;
      wsum += ok ? m_in->group_w[j] : 0.0;
    }
    if (!ok || std::fabs(wsum - 1.0) > 1e-12) {
      delete s;
      return RT_ERR_ARG;
    }
    const int Ag = G * Ab;
    gdir.resize(3 * (size_t)Ag);
    gwt.resize(Ag);
    s->col_of_angle.resize(Ag);
    s->group_w.assign(m_in->group_w, m_in->group_w + G);
    for (int k = 0; k < Ag; ++k) {
      const bool second = k >= G * Hb;
      const int kk = second ? k - G * Hb : k;
      const int j = kk / Hb, a = kk % Hb + (second ? Hb : 0);
      for (int d = 0; d < 3; ++d) gdir[3 * k + d] = m_in->angle_dir[3 * a + d];
      gwt[k] = m_in->group_w[j] * m_in->angle_w[a];
      s->col_of_angle[k] = j * Ab + a;
    }
    mx.n_angles = Ag;
    mx.angle_dir = gdir.data();
    mx.angle_w = gwt.data();
  } else if (m_in->n_angles > 0) {
    s->col_of_angle.resize(m_in->n_angles);
    for (int k = 0; k < m_in->n_angles; ++k) s->col_of_angle[k] = k;
  }
  int st = RT_OK;
  auto bail = [&](int code) {
    rt_destroy(s);
    return code;
  };
  if (!(p->cbar > 0) || !(p->c > 0) || !(p->a_rad >= 0) || !(p->gamma_gas > 1) ||
      !(p->r_gas > 0) || !(p->cfl > 0) || (p->precision != RT_FP32 && p->precision != RT_FP64) ||
      (p->integrator != RT_FIRST_ORDER && p->integrator != RT_VAN_LEER) ||
      (p->boost != 0 && p->boost != 1) || (p->gcl != 0 && p->gcl != 1) ||
      (p->gcl && p->integrator != RT_FIRST_ORDER) || !std::isfinite(p->beta_P) ||
      !std::isfinite(p->beta_J) || ((p->beta_P != 0 || p->beta_J != 0) && !(p->T_ref > 0)) ||
      !(p->beta_P >= -3.0) || (p->plain_launches != 0 && p->plain_launches != 1) ||
      (p->float_quartic != 0 && p->float_quartic != 1) || (p->hydro != 0 && p->hydro != 1) ||
      (p->hydro && (!m->face_offset || G > 1 || p->gcl || p->beta_P != 0.0 ||
                    p->beta_J != 0.0)) ||
      (p->integrator == RT_VAN_LEER && !m->face_offset))
    return bail(RT_ERR_ARG);
  s->params = *p;
  s->plain_launches = p->plain_launches != 0;
  if (s->params.newton_max_iter <= 0) s->params.newton_max_iter = 64;
  s->precision = p->precision;
  s->rsize = p->precision == RT_FP32 ? 4 : 8;
  s->stream = (cudaStream_t)stream;
  if ((st = check_mesh(s, m)) != RT_OK ||
      (p->precision == RT_FP32 && (st = check_float_range(s, m, p->cbar)) != RT_OK)) {
    // keep the message: callers of a failed create cannot query it, so print it
    fprintf(stderr, "rt_create: %s\n", s->err.c_str());
    return bail(st);
  }
  if (cudaGetDevice(&s->device) != cudaSuccess) return bail(RT_ERR_CUDA);
  const int64_t N = m->n_cells;
  const int A = m->n_angles;
  s->n_cells = N;
  s->n_faces = m->n_faces;
  s->nnz = m->cell_face_ptr[N];
  s->n_angles = A;
  s->cell_of = morton_order(N, m->cell_centroid);
  // within each block of the step kernel, most faces first: the lanes of a
  // warp then loop over similar face counts
  for (int64_t b0 = 0; b0 < N; b0 += rt::CPB) {
    auto first = s->cell_of.begin() + b0, last = s->cell_of.begin() + std::min(N, b0 + rt::CPB);
    std::stable_sort(first, last, [&](int64_t x, int64_t y) {
      return m->cell_face_ptr[x + 1] - m->cell_face_ptr[x] >
             m->cell_face_ptr[y + 1] - m->cell_face_ptr[y];
    });
  }
  std::vector<int64_t> slot_of(N);
  for (int64_t ic = 0; ic < N; ++ic) slot_of[s->cell_of[ic]] = ic;
  s->volume.assign(m->cell_volume, m->cell_volume + N);
  // Courant step (the paper defers its form to its hydro scheme; this is
  // dt = cfl * min V^(1/3) / (cbar + max |w| of the cell's faces))
  double best = INFINITY;
  for (int64_t c = 0; c < N; ++c) {
    double wmax = 0;
    if (m->face_w)
      for (int64_t k = m->cell_face_ptr[c]; k < m->cell_face_ptr[c + 1]; ++k) {
        int32_t e = m->cell_face_idx[k];
        int64_t f = e >= 0 ? e : -(int64_t)e - 1;
        const double *w = m->face_w + 3 * f;
        wmax = std::max(wmax, std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
      }
    best = std::min(best, std::cbrt(m->cell_volume[c]) / (p->cbar + wmax));
  }
  s->dt_cfl = p->cfl * best;
  if (m->face_w)
    for (int64_t k = 0; k < 3 * m->n_faces && !s->moving; ++k) s->moving = m->face_w[k] != 0.0;

  int r = (s->precision == RT_FP32) ? build_device_mesh<float>(s, m, slot_of)
                                    : build_device_mesh<double>(s, m, slot_of);
  if (r != RT_OK) return bail(r);
  if (p->hydro) {
    // the gas dynamics run on static faces
    if (s->moving) {
      fprintf(stderr, "rt_create: hydro = 1 needs a static mesh (face_w NULL or zero)\n");
      return bail(RT_ERR_ARG);
    }
    r = rt::hydro_setup(s, m);
    if (r != RT_OK) return bail(r);
  }
  s->integrator = p->integrator;
  if (s->integrator == RT_VAN_LEER) {
    r = (s->precision == RT_FP32) ? build_recon<float>(s, m) : build_recon<double>(s, m);
    if (r != RT_OK) return bail(r);
  }
  if (s->precision == RT_FP64) {
    // the FP64 flux-coefficient table: 8 A/2 bytes per directed face
    const cudaError_t e = rt::build_uface(s);
    if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA);
  }
  // float rows with A = 16 m (32 <= A <= 128) whose blocks' face slots fit
  // the step kernel's shared-memory stage take the quad layout
  s->quad_end = (s->precision == RT_FP32 && A % 16 == 0 && A >= 32 && A <= 128 &&
                 s->max_block_slots <= rt::STAGE_SLOTS)
                    ? 32 * (A / 32)
                    : 0;
  // dense rows (padding the quad rows to whole 128-byte lines measured no gain)
  s->row_stride = A;
  const size_t RS = (size_t)s->row_stride;
  std::vector<double> vol_int(N), dir64(3 * (size_t)A), wt64(A);
  std::vector<int32_t> angle_of(A);
  for (int64_t ic = 0; ic < N; ++ic) vol_int[ic] = m->cell_volume[s->cell_of[ic]];
  for (int q = 0; q < A; ++q) {
    const int a = angle_of_position(q, A / 2, s->quad_end);
    angle_of[q] = s->col_of_angle[a];  // the caller column of the position's angle
    for (int d = 0; d < 3; ++d) dir64[3 * q + d] = m->angle_dir[3 * a + d];
    wt64[q] = m->angle_w[a];
  }
#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return bail(cuda_fail(s, e_, #call)); \
  } while (0)
  CK(upload(s, &s->d_cell_of, s->cell_of));
  CK(upload(s, &s->d_volume, vol_int));
  CK(upload(s, &s->d_dir64, dir64));
  CK(upload(s, &s->d_wt64, wt64));
  CK(upload(s, &s->d_angle_of, angle_of));
  {
    std::vector<int32_t> pos_of(angle_of.size());
    for (size_t q = 0; q < angle_of.size(); ++q) pos_of[(size_t)angle_of[q]] = (int32_t)q;
    CK(upload(s, &s->d_pos_of, pos_of));
  }
  CK(dalloc(s, &s->d_gs, N));
  CK(dalloc(s, &s->d_gd, N));
  CK(dalloc(s, &s->d_kind, N));
  CK(dalloc(s, &s->d_aux, N));
  CK(dalloc(s, &s->d_bc_row, N));
  CK(dalloc(s, &s->d_ext, 4 * (size_t)N));
  if (s->integrator == RT_VAN_LEER) {  // stage-1 intensities and their gradients
    CK(dalloc_bytes(s, &s->d_Ihalf, (size_t)N * RS * s->rsize));
    CK(dalloc_bytes(s, &s->d_grad, 3 * (size_t)N * RS * s->rsize));
  }
  CK(dalloc_bytes(s, &s->d_cellv, 4 * (size_t)N * s->rsize));
  CK(cudaMemsetAsync(s->d_cellv, 0, 4 * (size_t)N * s->rsize, s->stream));
  CK(dalloc(s, &s->d_status, 1));
  CK(dalloc(s, &s->d_bad, 1));
  CK(dalloc(s, &s->d_out16, 16));
  s->scratch_len = (size_t)rt::totals_scratch_len(N);
  CK(dalloc(s, &s->d_scratch, s->scratch_len));
  CK(dalloc_bytes(s, &s->d_I[0], (size_t)N * RS * s->rsize));
  CK(dalloc_bytes(s, &s->d_I[1], (size_t)N * RS * s->rsize));
  CK(dalloc_bytes(s, &s->d_I0, RS * s->rsize));
  CK(cudaMemsetAsync(s->d_I0, 0, RS * s->rsize, s->stream));
  CK(cudaMemsetAsync(s->d_I[0], 0, (size_t)N * RS * s->rsize, s->stream));
  CK(cudaMemsetAsync(s->d_I[1], 0, (size_t)N * RS * s->rsize, s->stream));
  CK(cudaMemsetAsync(s->d_kind, 0, N, s->stream));
  CK(cudaMemsetAsync(s->d_aux, 0, sizeof(double2) * N, s->stream));
  CK(cudaMemsetAsync(s->d_bc_row, 0, sizeof(int32_t) * N, s->stream));
  CK(cudaMemsetAsync(s->d_ext, 0, sizeof(double) * 4 * N, s->stream));
  CK(cudaMemsetAsync(s->d_status, 0, sizeof(unsigned), s->stream));
  CK(cudaMemsetAsync(s->d_bad, 0xff, sizeof(unsigned long long), s->stream));
  s->n_rows = 1;
  // upwind positivity bound: a float screen over float slots (for double
  // states a temporary float copy), then the exact double sums of the
  // candidates
  rt::SlotF *fslot = reinterpret_cast<rt::SlotF *>(s->d_slot);
  if (s->precision == RT_FP64) {
    // a power of two that brings the largest cbar A and A |w| near 1, so
    // that the float screen neither overflows nor flushes at physical units
    double big = 0.0;
    for (int64_t f = 0; f < m->n_faces; ++f) {
      double v = p->cbar * m->face_area[f];
      if (m->face_w) {
        const double *w = m->face_w + 3 * f;
        v = std::max(v, m->face_area[f] * std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
      }
      big = std::max(big, v);
    }
    s->screen_scale = big > 0.0 ? std::ldexp(1.0, -std::ilogb(big)) : 1.0;
    std::vector<int64_t> p2;
    std::vector<int32_t> n2;
    std::vector<rt::SlotF> sf;
    std::vector<double> w2;
    std::vector<float> v2;
    fill_geometry<float>(s, m, slot_of, p2, n2, sf, w2, v2);
    fslot = nullptr;
    CK(cudaMalloc(&fslot, sf.size() * sizeof(rt::SlotF)));
    CK(cudaMemcpy(fslot, sf.data(), sf.size() * sizeof(rt::SlotF), cudaMemcpyHostToDevice));
  }
  if (p->gcl) {
    // geometric conservation law: sum_f A_f w_f . n_f per cell (outward
    // normals, faces in list order), and the per-cell factor of the
    // positivity limit that the step checks against the current volume
    std::vector<double> rate(N, 0.0);
    for (int64_t ic = 0; ic < N && m->face_w; ++ic) {
      const int64_t c = s->cell_of[ic];
      double r = 0.0;
      for (int64_t k = m->cell_face_ptr[c]; k < m->cell_face_ptr[c + 1]; ++k) {
        const int32_t e = m->cell_face_idx[k];
        const int64_t f = e >= 0 ? e : -(int64_t)e - 1;
        const double sgn = e >= 0 ? 1.0 : -1.0;
        const double *w = m->face_w + 3 * f, *nf = m->face_normal + 3 * f;
        r += m->face_area[f] * (sgn * (w[0] * nf[0] + w[1] * nf[1] + w[2] * nf[2]));
      }
      rate[ic] = r;
    }
    CK(upload(s, &s->d_gcl_rate, rate));
    CK(dalloc(s, &s->d_gcl_kv, N));
  }
  double kmax = 0;
  cudaError_t pe = rt::launch_positivity(s, fslot, s->d_out16, s->d_gcl_kv);
  if (pe == cudaSuccess)
    pe = cudaMemcpyAsync(&kmax, s->d_out16, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (pe == cudaSuccess) pe = cudaStreamSynchronize(s->stream);
  if (s->precision == RT_FP64) cudaFree(fslot);
  CK(pe);
#undef CK
  s->dt_max = kmax > 0 ? 1.0 / kmax : INFINITY;
  *out = s;
  return RT_OK;
}

int rt_set_gas(rt_state *s, const double *rho, const double *e, const double *m,
               const double *kP, const double *kJ, const double *kS) {
  if (!s) return RT_ERR_ARG;
  ++s->gen;  // captured step graphs may hold old arguments
  if (!rho || !e || !m || !kP || !kJ || !kS) return fail(s, RT_ERR_ARG, "rt_set_gas: NULL array");
  const int64_t N = s->n_cells;
  const int G = s->n_groups;  // opacity arrays hold G values per cell
  std::vector<rt::GasStatic> gs(N);
  std::vector<rt::GasDyn> gd(N);
  std::vector<double> kapg(G > 1 ? (size_t)N * G * 3 : 0);
  for (int64_t ic = 0; ic < N; ++ic) {
    const int64_t c = s->cell_of[ic];
    bool ok = rho[c] > 0 && std::isfinite(e[c]) && std::isfinite(m[3 * c]) &&
              std::isfinite(m[3 * c + 1]) && std::isfinite(m[3 * c + 2]);
    for (int j = 0; j < G; ++j) {
      const int64_t k = c * G + j;
      ok = ok && kP[k] >= 0 && kJ[k] >= 0 && kS[k] >= 0 && std::isfinite(kP[k] + kJ[k] + kS[k]);
    }
    if (!ok) return fail(s, RT_ERR_ARG, "rt_set_gas: rho must be > 0, opacities >= 0, all finite");
    const double rcv = rho[c] * s->params.r_gas / (s->params.gamma_gas - 1.0);
    if (s->precision == RT_FP32) {
      // float copies of rho kappa and rho c_v, and the float frame velocity
      // and internal energy, must not overflow
      bool fit = std::fabs(rcv) <= 0x1p125 && std::fabs(e[c]) <= 0x1p125 &&
                 std::fabs(m[3 * c] / rho[c]) <= 0x1p125 &&
                 std::fabs(m[3 * c + 1] / rho[c]) <= 0x1p125 &&
                 std::fabs(m[3 * c + 2] / rho[c]) <= 0x1p125;
      for (int j = 0; j < G; ++j) {
        const int64_t k = c * G + j;
        fit = fit && rho[c] * kP[k] <= 0x1p125 && rho[c] * kJ[k] <= 0x1p125 &&
              rho[c] * kS[k] <= 0x1p125;
      }
      if (!fit)
        return fail(s, RT_ERR_ARG,
                    "rt_set_gas: RT_FP32 state: rho kappa, rho c_v, e or v outside float range "
                    "(|x| <= 2^125); rescale the units or use RT_FP64");
    }
    const int64_t c0 = c * G;  // the grey record holds group 0's opacities
    gs[ic] = {rho[c], rho[c] * kP[c0], rho[c] * kJ[c0], rho[c] * kS[c0], 1.0 / rho[c], rcv,
              (float)(rho[c] * kP[c0]), (float)(rho[c] * kJ[c0]), (float)(rho[c] * kS[c0]),
              (float)rcv};
    gd[ic] = {e[c], m[3 * c], m[3 * c + 1], m[3 * c + 2]};
    for (int j = 0; j < G && G > 1; ++j) {
      double *k = &kapg[((size_t)ic * G + j) * 3];
      k[0] = rho[c] * kP[c * G + j];
      k[1] = rho[c] * kJ[c * G + j];
      k[2] = rho[c] * kS[c * G + j];
    }
  }
  if (G > 1) {
    std::vector<float> kapgf((size_t)N * G * 4, 0.0f);
    for (size_t i = 0; i < (size_t)N * G; ++i)
      for (int k = 0; k < 3; ++k) kapgf[4 * i + k] = (float)kapg[3 * i + k];
    if (!s->d_kapg) RT_CUDA(s, dalloc(s, &s->d_kapg, kapg.size()));
    if (!s->d_kapgf) RT_CUDA(s, dalloc(s, &s->d_kapgf, kapgf.size()));
    RT_CUDA(s, cudaMemcpy(s->d_kapg, kapg.data(), sizeof(double) * kapg.size(),
                          cudaMemcpyHostToDevice));
    RT_CUDA(s, cudaMemcpy(s->d_kapgf, kapgf.data(), sizeof(float) * kapgf.size(),
                          cudaMemcpyHostToDevice));
  }
  RT_CUDA(s, cudaMemcpyAsync(s->d_gs, gs.data(), sizeof(rt::GasStatic) * N, cudaMemcpyHostToDevice,
                             s->stream));
  RT_CUDA(s, cudaMemcpyAsync(s->d_gd, gd.data(), sizeof(rt::GasDyn) * N, cudaMemcpyHostToDevice,
                             s->stream));
  if (s->params.beta_J != 0.0) {
    // kappa_J follows the gas temperature: keep rho kappa_J at T_ref and
    // start from kappa_J(T^0)
    std::vector<double> rkJ0(N);
    for (int64_t ic = 0; ic < N; ++ic) rkJ0[ic] = gs[ic].rkJ;
    if (!s->d_rkJ0) RT_CUDA(s, dalloc(s, &s->d_rkJ0, N));
    RT_CUDA(s, cudaMemcpyAsync(s->d_rkJ0, rkJ0.data(), sizeof(double) * N, cudaMemcpyHostToDevice,
                               s->stream));
    RT_CUDA(s, cudaStreamSynchronize(s->stream));  // rkJ0 is a host temporary
    RT_CUDA(s, rt::launch_opacity_refresh(s));
  }
  if (s->params.hydro) {
    // the opacities per unit mass, for the coefficients after the density changes
    std::vector<double> km(3 * (size_t)N);
    for (int64_t ic = 0; ic < N; ++ic) {
      const int64_t c = s->cell_of[ic];
      km[3 * ic] = kP[c];
      km[3 * ic + 1] = kJ[c];
      km[3 * ic + 2] = kS[c];
    }
    RT_CUDA(s, cudaMemcpy(rt::hydro_kmass(s), km.data(), sizeof(double) * km.size(),
                          cudaMemcpyHostToDevice));
  }
  RT_CUDA(s, cudaMemsetAsync(s->d_ext, 0, sizeof(double) * 4 * N, s->stream));
  // per-cell frame velocity and rho (kJ + kS) in the state precision
  RT_CUDA(s, rt::launch_cellv(s));
  RT_CUDA(s, cudaMemsetAsync(s->d_status, 0, sizeof(unsigned), s->stream));
  RT_CUDA(s, cudaMemsetAsync(s->d_bad, 0xff, sizeof(unsigned long long), s->stream));
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  s->gas_set = true;
  return RT_OK;
}

int rt_set_gas_energy(rt_state *s, const double *e, const double *m, int on_device) {
  if (!s) return RT_ERR_ARG;
  if (!e || !m) return fail(s, RT_ERR_ARG, "rt_set_gas_energy: NULL array");
  if (!s->gas_set) return fail(s, RT_ERR_STATE, "rt_set_gas_energy before rt_set_gas");
  ++s->gen;  // captured step graphs may hold old arguments
  const int64_t N = s->n_cells;
  if (on_device) {
    RT_CUDA(s, rt::launch_gas_in(s, e, m));
  } else {
    std::vector<rt::GasDyn> gd(N);
    for (int64_t ic = 0; ic < N; ++ic) {
      const int64_t c = s->cell_of[ic];
      if (!std::isfinite(e[c]) || !std::isfinite(m[3 * c]) || !std::isfinite(m[3 * c + 1]) ||
          !std::isfinite(m[3 * c + 2]))
        return fail(s, RT_ERR_ARG, "rt_set_gas_energy: e and m must be finite");
      gd[ic] = {e[c], m[3 * c], m[3 * c + 1], m[3 * c + 2]};
    }
    RT_CUDA(s, cudaMemcpyAsync(s->d_gd, gd.data(), sizeof(rt::GasDyn) * N,
                               cudaMemcpyHostToDevice, s->stream));
    RT_CUDA(s, cudaStreamSynchronize(s->stream));  // gd is a host temporary
  }
  if (s->params.beta_J != 0.0) RT_CUDA(s, rt::launch_opacity_refresh(s));
  RT_CUDA(s, rt::launch_cellv(s));
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  return RT_OK;
}

int rt_set_cells(rt_state *s, const uint8_t *kind, const double *tau, const double *emit,
                 const double *isrc, const int32_t *bc_row, int64_t n_rows, const double *I0) {
  if (!s) return RT_ERR_ARG;
  ++s->gen;  // captured step graphs may hold old arguments
  const int64_t N = s->n_cells;
  const int A = s->n_angles;
  std::vector<uint8_t> k(N, 0);
  std::vector<double2> aux(N, double2{0, 0});
  std::vector<int32_t> row(N, 0);
  if (kind) {
    bool need_bc = false, need_em = false;
    for (int64_t c = 0; c < N; ++c) {
      if (kind[c] > 2) return fail(s, RT_ERR_ARG, "rt_set_cells: kind must be 0, 1 or 2");
      need_bc |= kind[c] == RT_CELL_BOUNDARY;
      need_em |= kind[c] == RT_CELL_EMITTER;
    }
    if (need_bc && (!tau || !bc_row || !I0 || n_rows < 1))
      return fail(s, RT_ERR_ARG, "rt_set_cells: boundary cells need tau, bc_row and I0");
    if (need_em && (!emit || !isrc))
      return fail(s, RT_ERR_ARG, "rt_set_cells: emitter cells need emit_rate and I_src");
    for (int64_t ic = 0; ic < N; ++ic) {
      const int64_t c = s->cell_of[ic];
      k[ic] = kind[c];
      if (kind[c] == RT_CELL_BOUNDARY) {
        if (bc_row[c] < 0 || bc_row[c] >= n_rows || !(tau[c] >= 0))
          return fail(s, RT_ERR_ARG, "rt_set_cells: bad bc_row or negative tau");
        aux[ic] = double2{tau[c], 0.0};
        row[ic] = bc_row[c];
      } else if (kind[c] == RT_CELL_EMITTER) {
        if (!(emit[c] >= 0) || !std::isfinite(isrc[c]))
          return fail(s, RT_ERR_ARG, "rt_set_cells: bad emitter rate or intensity");
        aux[ic] = double2{emit[c], isrc[c]};
      }
    }
  }
  RT_CUDA(s, cudaMemcpyAsync(s->d_kind, k.data(), N, cudaMemcpyHostToDevice, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(s->d_aux, aux.data(), sizeof(double2) * N, cudaMemcpyHostToDevice,
                             s->stream));
  RT_CUDA(s, cudaMemcpyAsync(s->d_bc_row, row.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice,
                             s->stream));
  if (kind && I0 && n_rows >= 1) {
    RT_CUDA(s, cudaStreamSynchronize(s->stream));
    if (n_rows != s->n_rows) {
      cudaFree(s->d_I0);
      s->d_I0 = nullptr;
      RT_CUDA(s, dalloc_bytes(s, &s->d_I0, (size_t)n_rows * s->row_stride * s->rsize));
      s->n_rows = n_rows;
    }
    // rows in the internal angle order, row_stride reals apart (padding zero)
    const int64_t RS = s->row_stride;
    std::vector<double> rows((size_t)n_rows * RS, 0.0);
    for (int64_t r = 0; r < n_rows; ++r)
      for (int q = 0; q < A; ++q)
        rows[r * RS + q] = I0[r * A + s->col_of_angle[angle_of_position(q, A / 2, s->quad_end)]];
    if (s->precision == RT_FP32) {
      std::vector<float> f(rows.begin(), rows.end());
      RT_CUDA(s, cudaMemcpy(s->d_I0, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    } else {
      RT_CUDA(s, cudaMemcpy(s->d_I0, rows.data(), rows.size() * 8, cudaMemcpyHostToDevice));
    }
  }
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  return RT_OK;
}

// The device-side address of page-locked (cudaHostAlloc / cudaHostRegister)
// host memory, which kernels may read and write; NULL for any other pointer
// (pageable memory then goes through a staged copy).
// The device address of page-locked host memory [p, p + bytes), or NULL if
// any of it is not page-locked: the driver reports the registered range that
// holds p, and the whole span must lie in it (a buffer registered in part
// takes the staged copy).
static const void *pinned_device_address(const void *p, size_t bytes) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  using GetAttr = CUresult (*)(void *, CUpointer_attribute, CUdeviceptr);
  static GetAttr get = reinterpret_cast<GetAttr>(rt::driver_fn("cuPointerGetAttribute"));
  if (!get) return nullptr;
  CUdeviceptr start = 0;
  size_t size = 0;
  if (get(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)(uintptr_t)p) !=
          CUDA_SUCCESS ||
      get(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)(uintptr_t)p) != CUDA_SUCCESS)
    return nullptr;
  const uintptr_t a = (uintptr_t)p, lo = (uintptr_t)start;
  if (a < lo || a - lo > size || bytes > size - (a - lo)) return nullptr;
  return at.devicePointer;
}

int rt_set_intensity(rt_state *s, const void *I, int on_device) {
  if (!s || !I) return s ? fail(s, RT_ERR_ARG, "rt_set_intensity: NULL") : RT_ERR_ARG;
  ++s->gen;  // captured step graphs may hold old arguments
  const size_t bytes = (size_t)s->n_cells * s->n_angles * s->rsize;
  const void *src = I;
  void *stage = s->d_I[s->cur ^ 1];
  if (!on_device) {
    if (const void *dev = pinned_device_address(I, bytes)) {
      // page-locked host rows: one pass reads them over the host link and
      // writes the internal rows
      RT_CUDA(s, rt::launch_permute_in_host(s, dev, s->d_I[s->cur], s->row_stride));
      RT_CUDA(s, cudaStreamSynchronize(s->stream));
      return RT_OK;
    }
    RT_CUDA(s, cudaMemcpyAsync(stage, I, bytes, cudaMemcpyHostToDevice, s->stream));
    src = stage;
  }
  RT_CUDA(s, rt::launch_permute_in(s, src, s->d_I[s->cur], s->row_stride));
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  return RT_OK;
}

int rt_get_intensity(rt_state *s, void *I, int on_device) {
  if (!s || !I) return s ? fail(s, RT_ERR_ARG, "rt_get_intensity: NULL") : RT_ERR_ARG;
  const size_t bytes = (size_t)s->n_cells * s->n_angles * s->rsize;
  if (on_device) {
    RT_CUDA(s, rt::launch_permute_out(s, s->d_I[s->cur], I, s->row_stride));
  } else if (void *dev = const_cast<void *>(pinned_device_address(I, bytes))) {
    RT_CUDA(s, rt::launch_permute_out_host(s, s->d_I[s->cur], dev, s->row_stride));
  } else {
    void *stage = s->d_I[s->cur ^ 1];
    RT_CUDA(s, rt::launch_permute_out(s, s->d_I[s->cur], stage, s->row_stride));
    RT_CUDA(s, cudaMemcpyAsync(I, stage, bytes, cudaMemcpyDeviceToHost, s->stream));
  }
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  return RT_OK;
}

int rt_get_gas(rt_state *s, double *e, double *m, double *ext, int on_device) {
  if (!s) return RT_ERR_ARG;
  const int64_t N = s->n_cells;
  if (on_device) {
    RT_CUDA(s, rt::launch_gas_out(s, e, m, ext));
    RT_CUDA(s, cudaStreamSynchronize(s->stream));
    return RT_OK;
  }
  double *de = nullptr, *dm = nullptr, *dx = nullptr;
  // staging in the idle intensity buffer when it is large enough, else allocate
  const size_t need = sizeof(double) * 8 * (size_t)N;
  const size_t have = (size_t)N * s->n_angles * s->rsize;
  void *tmp = nullptr;
  bool own = false;
  if (have >= need) {
    tmp = s->d_I[s->cur ^ 1];
  } else {
    RT_CUDA(s, cudaMalloc(&tmp, need));
    own = true;
  }
  de = (double *)tmp;
  dm = de + N;
  dx = dm + 3 * N;
  cudaError_t err = rt::launch_gas_out(s, e ? de : nullptr, m ? dm : nullptr, ext ? dx : nullptr);
  if (err == cudaSuccess && e) err = cudaMemcpyAsync(e, de, 8 * N, cudaMemcpyDeviceToHost, s->stream);
  if (err == cudaSuccess && m)
    err = cudaMemcpyAsync(m, dm, 24 * N, cudaMemcpyDeviceToHost, s->stream);
  if (err == cudaSuccess && ext)
    err = cudaMemcpyAsync(ext, dx, 32 * N, cudaMemcpyDeviceToHost, s->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s->stream);
  if (own) cudaFree(tmp);
  if (err != cudaSuccess) return cuda_fail(s, err, "rt_get_gas");
  return RT_OK;
}

int rt_dt_limits(rt_state *s, double *dt_cfl, double *dt_max) {
  if (!s) return RT_ERR_ARG;
  if (dt_cfl) *dt_cfl = s->dt_cfl;
  if (dt_max) *dt_max = s->dt_max;
  return RT_OK;
}

// The graph of RT_GRAPH_STEPS steps from the current buffer parity at dt,
// captured now if the cached one is missing or stale.  An even number of
// steps brings the buffers back, so the graph can be replayed any number of
// times.  Capturing runs the launch code on the host without executing the
// kernels: the buffer index and the launch count are restored afterwards.
static cudaError_t step_graph(rt_state *s, double dt, cudaGraphExec_t *out) {
  static_assert(RT_GRAPH_STEPS % 2 == 0, "the graph must bring the buffers back");
  const int par = s->cur;
  if (s->graph[par] && s->graph_dt[par] == dt && s->graph_gen[par] == s->gen) {
    *out = s->graph[par];
    return cudaSuccess;
  }
  if (s->graph[par]) {
    cudaGraphExecDestroy(s->graph[par]);
    s->graph[par] = nullptr;
  }
  // captured on a stream of the state's own (the caller's stream may be the
  // legacy default stream, which cannot be captured); replayed on the
  // caller's stream
  if (!s->cap_stream) {
    const cudaError_t ec = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
    if (ec != cudaSuccess) return ec;
  }
  const int64_t l0 = s->launches;
  cudaStream_t user = s->stream;
  s->stream = s->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    s->stream = user;
    return e;
  }
  for (int i = 0; i < RT_GRAPH_STEPS && e == cudaSuccess; ++i) e = rt::launch_step(s, dt);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
  s->stream = user;
  s->cur = par;
  const int64_t per = s->launches - l0;
  s->launches = l0;
  if (e == cudaSuccess) e = e2;
  cudaGraphExec_t x = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) return e;
  s->graph[par] = x;
  s->graph_dt[par] = dt;
  s->graph_gen[par] = s->gen;
  s->graph_launches[par] = per;
  *out = x;
  return cudaSuccess;
}

static int launch_steps(rt_state *s, int32_t n, double dt, double *dt_used, bool sync) {
  if (!s) return RT_ERR_ARG;
  if (!s->gas_set) return fail(s, RT_ERR_STATE, "rt_set_gas must be called before stepping");
  if (n < 0) return fail(s, RT_ERR_ARG, "negative step count");
  if (!(dt > 0)) dt = s->dt_cfl;
  if (!std::isfinite(dt)) return fail(s, RT_ERR_ARG, "dt must be finite");
  if (dt > s->dt_max) {
    char buf[160];
    snprintf(buf, sizeof buf, "dt = %.6g exceeds the upwind positivity limit %.6g", dt, s->dt_max);
    return fail(s, RT_ERR_CFL, buf);
  }
  if (dt_used) *dt_used = dt;
  int32_t left = n;
  if (!s->plain_launches && n >= RT_GRAPH_STEPS) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s->stream) RT_CUDA(s, cudaStreamIsCapturing(s->stream, &cs));
    cudaGraphExec_t x = nullptr;
    if (cs == cudaStreamCaptureStatusNone && step_graph(s, dt, &x) != cudaSuccess) {
      // no graph on this device or stream: plain launches from now on
      (void)cudaGetLastError();
      s->plain_launches = true;
      x = nullptr;
    }
    if (x) {
      for (; left >= RT_GRAPH_STEPS; left -= RT_GRAPH_STEPS) {
        RT_CUDA(s, cudaGraphLaunch(x, s->stream));
        s->launches += s->graph_launches[s->cur];
      }
    }
  }
  for (; left > 0; --left) RT_CUDA(s, rt::launch_step(s, dt));
  return sync ? sync_status(s) : RT_OK;
}

int rt_step(rt_state *s, double dt, double *dt_used) {
  return launch_steps(s, 1, dt, dt_used, true);
}

int rt_step_io(rt_state *s, double dt, const void *I_in, void *I_out) {
  if (!s || !I_in || !I_out) return s ? fail(s, RT_ERR_ARG, "rt_step_io: NULL") : RT_ERR_ARG;
  if (!s->gas_set) return fail(s, RT_ERR_STATE, "rt_set_gas must be called before stepping");
  if (!(dt > 0)) dt = s->dt_cfl;
  if (!std::isfinite(dt)) return fail(s, RT_ERR_ARG, "dt must be finite");
  if (dt > s->dt_max) return fail(s, RT_ERR_CFL, "rt_step_io: dt exceeds the upwind positivity limit");
  const size_t bytes = (size_t)s->n_cells * s->n_angles * s->rsize;
  if (!pinned_device_address(I_in, bytes) || !pinned_device_address(I_out, bytes))
    return fail(s, RT_ERR_ARG, "rt_step_io: I_in and I_out must be page-locked host memory in full");
  if (!s->io_in) {
    RT_CUDA(s, dalloc_bytes(s, &s->d_io_in, bytes));
    RT_CUDA(s, dalloc_bytes(s, &s->d_io_out, bytes));
    RT_CUDA(s, cudaStreamCreateWithFlags(&s->io_in, cudaStreamNonBlocking));
    RT_CUDA(s, cudaStreamCreateWithFlags(&s->io_out, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&s->ev_h2d, &s->ev_pin, &s->ev_pout, &s->ev_d2h})
      RT_CUDA(s, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    // nothing staged yet: both staging arrays are free after the work queued so far
    RT_CUDA(s, cudaEventRecord(s->ev_pin, s->stream));
    RT_CUDA(s, cudaEventRecord(s->ev_d2h, s->stream));
  }
  ++s->gen;  // the rows change outside the captured step graphs
  // in: host rows -> staging (copy engine), once the previous call's device
  // permute has read the staging array; it overlaps that call's step and
  // result copy
  RT_CUDA(s, cudaStreamWaitEvent(s->io_in, s->ev_pin, 0));
  RT_CUDA(s, cudaMemcpyAsync(s->d_io_in, I_in, bytes, cudaMemcpyHostToDevice, s->io_in));
  RT_CUDA(s, cudaEventRecord(s->ev_h2d, s->io_in));
  // the state's stream: staging -> internal rows, the step, internal rows ->
  // the result staging (once the previous result has been copied out)
  RT_CUDA(s, cudaStreamWaitEvent(s->stream, s->ev_h2d, 0));
  RT_CUDA(s, rt::launch_permute_in(s, s->d_io_in, s->d_I[s->cur], s->row_stride));
  RT_CUDA(s, cudaEventRecord(s->ev_pin, s->stream));
  RT_CUDA(s, rt::launch_step(s, dt));
  RT_CUDA(s, cudaStreamWaitEvent(s->stream, s->ev_d2h, 0));
  RT_CUDA(s, rt::launch_permute_out(s, s->d_I[s->cur], s->d_io_out, s->row_stride));
  RT_CUDA(s, cudaEventRecord(s->ev_pout, s->stream));
  // out: result staging -> host rows (copy engine), overlapping the next
  // call's input copy and step
  RT_CUDA(s, cudaStreamWaitEvent(s->io_out, s->ev_pout, 0));
  RT_CUDA(s, cudaMemcpyAsync(I_out, s->d_io_out, bytes, cudaMemcpyDeviceToHost, s->io_out));
  RT_CUDA(s, cudaEventRecord(s->ev_d2h, s->io_out));
  return RT_OK;
}

int rt_run(rt_state *s, int32_t n, double dt, double *dt_used) {
  return launch_steps(s, n, dt, dt_used, true);
}

int rt_launch(rt_state *s, int32_t n, double dt, double *dt_used) {
  return launch_steps(s, n, dt, dt_used, false);
}

static int hydro_ready(rt_state *s, const char *who) {
  if (!s->params.hydro) {
    std::string m = std::string(who) + ": the state was created without hydro = 1";
    return fail(s, RT_ERR_STATE, m.c_str());
  }
  if (!s->gas_set) {
    std::string m = std::string(who) + ": rt_set_gas must be called first";
    return fail(s, RT_ERR_STATE, m.c_str());
  }
  return RT_OK;
}

int rt_hydro_step(rt_state *s, double dt, int32_t order) {
  if (!s) return RT_ERR_ARG;
  int st = hydro_ready(s, "rt_hydro_step");
  if (st != RT_OK) return st;
  if (!(dt > 0) || !std::isfinite(dt)) return fail(s, RT_ERR_ARG, "rt_hydro_step: dt must be positive and finite");
  if (order != 1 && order != 2) return fail(s, RT_ERR_ARG, "rt_hydro_step: order must be 1 or 2");
  RT_CUDA(s, rt::launch_hydro_step(s, dt, order));
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  unsigned bad = 0;
  RT_CUDA(s, cudaMemcpy(&bad, s->d_status, sizeof bad, cudaMemcpyDeviceToHost));
  if (bad & rt::ST_NONFINITE) {
    unsigned long long c = 0;
    RT_CUDA(s, cudaMemcpy(&c, s->d_bad, sizeof c, cudaMemcpyDeviceToHost));
    char buf[160];
    snprintf(buf, sizeof buf, "rt_hydro_step: non-positive density or pressure (first cell %lld)",
             c < (unsigned long long)s->n_cells ? (long long)s->cell_of[c] : -1LL);
    return fail(s, RT_ERR_NONFINITE, buf);
  }
  return RT_OK;
}

int rt_hydro_dt(rt_state *s, double cfl, double *dt) {
  if (!s || !dt) return s ? fail(s, RT_ERR_ARG, "rt_hydro_dt: NULL") : RT_ERR_ARG;
  int st = hydro_ready(s, "rt_hydro_dt");
  if (st != RT_OK) return st;
  if (!(cfl > 0) || !std::isfinite(cfl)) return fail(s, RT_ERR_ARG, "rt_hydro_dt: cfl must be positive");
  RT_CUDA(s, rt::launch_hydro_dt(s, cfl, dt));
  return RT_OK;
}

int rt_radhydro_step(rt_state *s, double dt, int32_t n_sub, int32_t order, double *dt_rad) {
  if (!s) return RT_ERR_ARG;
  if (n_sub < 1) return fail(s, RT_ERR_ARG, "rt_radhydro_step: n_sub must be >= 1");
  int st = rt_hydro_step(s, dt, order);
  if (st != RT_OK) return st;
  return launch_steps(s, n_sub, dt / n_sub, dt_rad, true);
}

int rt_get_density(rt_state *s, double *rho, int on_device) {
  if (!s || !rho) return s ? fail(s, RT_ERR_ARG, "rt_get_density: NULL") : RT_ERR_ARG;
  const int64_t N = s->n_cells;
  if (on_device) {
    RT_CUDA(s, rt::launch_density_out(s, rho));
  } else {
    double *buf = nullptr;
    RT_CUDA(s, cudaMalloc((void **)&buf, sizeof(double) * N));
    cudaError_t e = rt::launch_density_out(s, buf);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rho, buf, sizeof(double) * N, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(s, e, "rt_get_density");
  }
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  return RT_OK;
}

int rt_moments(rt_state *s, double *E, double *F, double *P, int on_device) {
  if (!s) return RT_ERR_ARG;
  const int64_t N = s->n_cells;
  if (on_device) {
    RT_CUDA(s, rt::launch_moments(s, E, F, P));
    RT_CUDA(s, cudaStreamSynchronize(s->stream));
    return RT_OK;
  }
  double *buf = nullptr;
  RT_CUDA(s, cudaMalloc((void **)&buf, sizeof(double) * 10 * N));
  double *dE = buf, *dF = buf + N, *dP = buf + 4 * N;
  cudaError_t err = rt::launch_moments(s, E ? dE : nullptr, F ? dF : nullptr, P ? dP : nullptr);
  if (err == cudaSuccess && E) err = cudaMemcpyAsync(E, dE, 8 * N, cudaMemcpyDeviceToHost, s->stream);
  if (err == cudaSuccess && F) err = cudaMemcpyAsync(F, dF, 24 * N, cudaMemcpyDeviceToHost, s->stream);
  if (err == cudaSuccess && P) err = cudaMemcpyAsync(P, dP, 48 * N, cudaMemcpyDeviceToHost, s->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s->stream);
  cudaFree(buf);
  if (err != cudaSuccess) return cuda_fail(s, err, "rt_moments");
  return RT_OK;
}

int rt_totals(rt_state *s, double out[16]) {
  if (!s || !out) return s ? fail(s, RT_ERR_ARG, "rt_totals: NULL") : RT_ERR_ARG;
  RT_CUDA(s, rt::launch_totals(s, s->d_out16));
  RT_CUDA(s, cudaMemcpyAsync(out, s->d_out16, sizeof(double) * 16, cudaMemcpyDeviceToHost, s->stream));
  return sync_status(s);
}

int rt_sync(rt_state *s) {
  if (!s) return RT_ERR_ARG;
  return sync_status(s);
}

int rt_adjoint_step(rt_state *s, double dt, const void *I_n, const double *e_n, const double *m_n,
                    const void *lam_I1, const double *lam_e1, const double *lam_m1, void *lam_I,
                    double *lam_e, double *lam_m, double *grad_kappa_P, double *grad_kappa_J,
                    int on_device) {
  if (!s) return RT_ERR_ARG;
  if (!s->gas_set) return fail(s, RT_ERR_STATE, "rt_set_gas must be called before the adjoint");
  if (s->integrator != RT_FIRST_ORDER)
    return fail(s, RT_ERR_STATE, "rt_adjoint_step reverses the first-order step only");
  if (s->params.boost)
    return fail(s, RT_ERR_STATE,
                "rt_adjoint_step reverses the first-order comoving transformation only");
  if (s->params.gcl)
    return fail(s, RT_ERR_STATE, "rt_adjoint_step reverses steps on fixed cell volumes only");
  if (s->params.beta_P != 0.0 || s->params.beta_J != 0.0)
    return fail(s, RT_ERR_STATE, "rt_adjoint_step reverses steps with constant opacities only");
  if (s->n_groups > 1)
    return fail(s, RT_ERR_STATE, "rt_adjoint_step reverses grey steps only");
  if (!I_n || !e_n || !m_n || !lam_I1 || !lam_e1 || !lam_m1 || !lam_I || !lam_e || !lam_m ||
      !grad_kappa_P || !grad_kappa_J)
    return fail(s, RT_ERR_ARG, "rt_adjoint_step: NULL argument");
  if (!(dt > 0)) dt = s->dt_cfl;
  if (!std::isfinite(dt) || dt > s->dt_max) return fail(s, RT_ERR_CFL, "rt_adjoint_step: bad dt");
  const int64_t N = s->n_cells;
  const size_t nI = (size_t)N * s->n_angles * s->rsize;
  if (!s->d_adj[0]) {
    for (int k = 0; k < 8; ++k) RT_CUDA(s, dalloc_bytes(s, &s->d_adj[k], nI));
    RT_CUDA(s, dalloc(s, &s->d_adj_ws, 25 * (size_t)N));
    RT_CUDA(s, dalloc(s, &s->d_adj_stage, 10 * (size_t)N));
  }
  if (on_device) {
    RT_CUDA(s, rt::adjoint_step(s, dt, I_n, e_n, m_n, lam_I1, lam_e1, lam_m1, lam_I, lam_e, lam_m,
                                grad_kappa_P, grad_kappa_J));
    RT_CUDA(s, cudaStreamSynchronize(s->stream));
    return RT_OK;
  }
  // host buffers: stage through device copies in the caller's order
  double *st = s->d_adj_stage;  // e, m(3), le1, lm1(3), gP, gJ; outputs reuse e / m / le1
  double *de = st, *dm = st + N, *dle1 = st + 4 * N, *dlm1 = st + 5 * N, *dgP = st + 8 * N,
         *dgJ = st + 9 * N;
  const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
  RT_CUDA(s, cudaMemcpyAsync(s->d_adj[5], I_n, nI, h2d, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(s->d_adj[6], lam_I1, nI, h2d, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(de, e_n, 8 * N, h2d, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(dm, m_n, 24 * N, h2d, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(dle1, lam_e1, 8 * N, h2d, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(dlm1, lam_m1, 24 * N, h2d, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(dgP, grad_kappa_P, 8 * N, h2d, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(dgJ, grad_kappa_J, 8 * N, h2d, s->stream));
  // outputs: lam_I -> d_adj[7]; lam_e, lam_m overwrite the staging of lam_e1, lam_m1
  // (each cell's are read by the thread that then writes the cell's outputs)
  RT_CUDA(s, rt::adjoint_step(s, dt, s->d_adj[5], de, dm, s->d_adj[6], dle1, dlm1, s->d_adj[7],
                              dle1, dlm1, dgP, dgJ));
  RT_CUDA(s, cudaMemcpyAsync(lam_I, s->d_adj[7], nI, d2h, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(lam_e, dle1, 8 * N, d2h, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(lam_m, dlm1, 24 * N, d2h, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(grad_kappa_P, dgP, 8 * N, d2h, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(grad_kappa_J, dgJ, 8 * N, d2h, s->stream));
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  return RT_OK;
}

int rt_get_state(rt_state *s, void *buf, size_t *bytes) {
  if (!s || !bytes) return RT_ERR_ARG;
  const int64_t N = s->n_cells;
  const size_t nI = (size_t)N * s->row_stride * s->rsize;  // internal rows with padding
  const size_t nV = s->params.gcl ? sizeof(double) * N : 0;   // the evolved volumes
  const size_t need = 64 + nI + sizeof(rt::GasDyn) * N + 32 * (size_t)N + nV;
  if (!buf) {
    *bytes = need;
    return RT_OK;
  }
  if (*bytes < need) return fail(s, RT_ERR_ARG, "rt_get_state: buffer too small");
  char *b = (char *)buf;
  int64_t hdr[8] = {0x52544742, N, s->n_angles, s->precision, (int64_t)nI, s->params.gcl, 0, 0};
  std::memcpy(b, hdr, 64);
  // internal order is fine: the state is restored into the same mesh
  RT_CUDA(s, cudaMemcpyAsync(b + 64, s->d_I[s->cur], nI, cudaMemcpyDeviceToHost, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(b + 64 + nI, s->d_gd, sizeof(rt::GasDyn) * N, cudaMemcpyDeviceToHost,
                             s->stream));
  RT_CUDA(s, cudaMemcpyAsync(b + 64 + nI + sizeof(rt::GasDyn) * N, s->d_ext, 32 * (size_t)N,
                             cudaMemcpyDeviceToHost, s->stream));
  if (nV)
    RT_CUDA(s, cudaMemcpyAsync(b + 64 + nI + sizeof(rt::GasDyn) * N + 32 * (size_t)N, s->d_volume,
                               nV, cudaMemcpyDeviceToHost, s->stream));
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  *bytes = need;
  return RT_OK;
}

int rt_set_state(rt_state *s, const void *buf, size_t bytes) {
  if (!s || !buf) return RT_ERR_ARG;
  ++s->gen;  // captured step graphs may hold old arguments
  const int64_t N = s->n_cells;
  const size_t nI = (size_t)N * s->row_stride * s->rsize;
  const size_t nV = s->params.gcl ? sizeof(double) * N : 0;
  const size_t need = 64 + nI + sizeof(rt::GasDyn) * N + 32 * (size_t)N + nV;
  int64_t hdr[8];
  if (bytes < need) return fail(s, RT_ERR_ARG, "rt_set_state: buffer too small");
  std::memcpy(hdr, buf, 64);
  if (hdr[0] != 0x52544742 || hdr[1] != N || hdr[2] != s->n_angles || hdr[3] != s->precision ||
      hdr[4] != (int64_t)nI || hdr[5] != s->params.gcl)
    return fail(s, RT_ERR_ARG, "rt_set_state: buffer does not match this state");
  const char *b = (const char *)buf;
  RT_CUDA(s, cudaMemcpyAsync(s->d_I[s->cur], b + 64, nI, cudaMemcpyHostToDevice, s->stream));
  RT_CUDA(s, cudaMemcpyAsync(s->d_gd, b + 64 + nI, sizeof(rt::GasDyn) * N, cudaMemcpyHostToDevice,
                             s->stream));
  RT_CUDA(s, cudaMemcpyAsync(s->d_ext, b + 64 + nI + sizeof(rt::GasDyn) * N, 32 * (size_t)N,
                             cudaMemcpyHostToDevice, s->stream));
  if (nV) {
    RT_CUDA(s, cudaMemcpyAsync(s->d_volume, b + 64 + nI + sizeof(rt::GasDyn) * N + 32 * (size_t)N,
                               nV, cudaMemcpyHostToDevice, s->stream));
    RT_CUDA(s, rt::launch_inv_vol(s));
  }
  RT_CUDA(s, rt::launch_opacity_refresh(s));  // kappa_J at the restored temperatures
  RT_CUDA(s, rt::launch_cellv(s));
  RT_CUDA(s, cudaStreamSynchronize(s->stream));
  return RT_OK;
}

int rt_device_bytes(const rt_state *s, size_t *bytes) {
  if (!s || !bytes) return RT_ERR_ARG;
  *bytes = s->device_bytes;
  return RT_OK;
}

int64_t rt_launch_count(const rt_state *s) { return s ? s->launches : -1; }

const char *rt_last_error(const rt_state *s) { return s ? s->err.c_str() : "null state"; }

void rt_destroy(rt_state *s) {
  if (!s) return;
  if (s->stream || true) cudaStreamSynchronize(s->stream);
  for (int k = 0; k < 2; ++k)
    if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  for (cudaStream_t st : {s->io_in, s->io_out})
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (cudaEvent_t e : {s->ev_h2d, s->ev_pin, s->ev_pout, s->ev_d2h})
    if (e) cudaEventDestroy(e);
  if (s->d_io_in) cudaFree(s->d_io_in);
  if (s->d_io_out) cudaFree(s->d_io_out);
  for (int k = 0; k < 8; ++k)
    if (s->d_adj[k]) cudaFree(s->d_adj[k]);
  if (s->d_adj_ws) cudaFree(s->d_adj_ws);
  if (s->d_adj_stage) cudaFree(s->d_adj_stage);
  void *bufs[] = {s->d_hface, s->d_hslot, s->d_hlsq, s->d_hwork, s->d_kapgf, s->d_kapg, s->d_rkJ0, s->d_gcl_rate, s->d_gcl_kv, s->d_recon, s->d_lsq, s->d_Ihalf, s->d_grad, s->d_uface, s->d_slot_nb, s->d_wface, s->d_angle_of, s->d_pos_of, s->d_cellv, s->d_ptr, s->d_nbr, s->d_slot, s->d_inv_vol, s->d_cell_of, s->d_volume, s->d_gs,
                  s->d_gd, s->d_kind, s->d_aux, s->d_bc_row, s->d_I0, s->d_ext, s->d_dir, s->d_wt,
                  s->d_dir64, s->d_wt64, s->d_I[0], s->d_I[1], s->d_status, s->d_bad,
                  s->d_scratch, s->d_out16};
  for (void *b : bufs)
    if (b) cudaFree(b);
  delete s;
}

}  // extern "C"
