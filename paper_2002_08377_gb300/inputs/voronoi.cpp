// Periodic Voronoi tessellation of a jittered lattice, built on the host.
//
// The mesh is an INPUT of the radiation step (Sec. 2: cells are the Voronoi
// cells of the mesh-generating points, faces carry area A_ij, unit normal
// i -> j and centroid r_ij).  Nothing here belongs to the radiation method;
// both the CPU oracle and the CUDA path take these arrays as given.
//
// Method: every cell is a convex polyhedron obtained by clipping a box around
// its generator with the bisector half-spaces of candidate neighbours, taken
// in order of increasing lattice distance.  The search stops once no further
// candidate can reach the cell (the "security radius": a plane at distance
// d/2 from the generator cannot cut a cell whose farthest vertex is closer
// than d/2).  Generators are lattice points plus a bounded jitter, so a lower
// bound on every candidate's distance is known from its lattice offset.
//
// Output conventions
//   faces are stored once, for the pair (i, j, image shift) with j > i, or
//   j == i and the image shift lexicographically positive (a cell meeting
//   its own periodic image, only possible on lattices 2 cells wide);
//   face_normal is the unit vector from generator i to (the image of) j;
//   face_centroid is expressed in the periodic frame of cell i;
//   the CSR of each cell lists its faces in increasing face index, entry f
//   (>= 0) when the cell is the face's first cell and -(f+1) when it is
//   the second cell.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Neighbour tag of a polyhedron face: generator j seen through image shift.
struct Tag {
  int32_t j;      // -1 for a wall of the initial box
  int8_t s[3];    // image shift in box lengths
};

// Convex polyhedron: vertices plus faces given as vertex loops, counter-
// clockwise seen from outside.
struct Poly {
  std::vector<V3> v;
  std::vector<std::vector<int>> f;
  std::vector<Tag> tag;
};

void make_box(Poly& p, V3 c, V3 h) {
  p.v.clear();
  p.f.clear();
  p.tag.clear();
  for (int k = 0; k < 8; ++k)
    p.v.push_back({c.x + ((k & 1) ? h.x : -h.x), c.y + ((k & 2) ? h.y : -h.y),
                   c.z + ((k & 4) ? h.z : -h.z)});
  // outward CCW loops of the six walls
  const int loops[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4},
                           {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};
  for (auto& l : loops) {
    p.f.push_back({l[0], l[1], l[2], l[3]});
    p.tag.push_back({-1, {0, 0, 0}});
  }
}

// Keep the half-space {x : dot(n, x) <= d}; the new face gets tag t.
// Returns false if the plane does not cut the polyhedron.
bool clip(Poly& p, V3 n, double d, Tag t, std::vector<double>& sd,
          std::vector<int>& remap) {
  const int nv = (int)p.v.size();
  sd.resize(nv);
  double scale = 0.0;
  bool any_out = false;
  for (int k = 0; k < nv; ++k) {
    sd[k] = dot(n, p.v[k]) - d;
    scale = std::max(scale, std::fabs(sd[k]));
  }
  const double eps = 1e-14 * (scale + std::fabs(d)) + 1e-300;
  for (int k = 0; k < nv; ++k) {
    if (sd[k] > eps) any_out = true;
    else if (sd[k] > 0) sd[k] = 0;  // on the plane: keep as inside
  }
  if (!any_out) return false;
  // new vertex list: kept vertices, then one vertex per cut edge
  remap.assign(nv, -1);
  std::vector<V3> nvtx;
  nvtx.reserve(nv + 8);
  for (int k = 0; k < nv; ++k)
    if (sd[k] <= 0) {
      remap[k] = (int)nvtx.size();
      nvtx.push_back(p.v[k]);
    }
  // cut vertices keyed by the (ordered) edge
  std::vector<std::pair<uint64_t, int>> cuts;
  auto cut_vertex = [&](int a, int b) -> int {
    uint64_t key = a < b ? ((uint64_t)a << 32) | (uint32_t)b
                         : ((uint64_t)b << 32) | (uint32_t)a;
    for (auto& c : cuts)
      if (c.first == key) return c.second;
    double ta = sd[a] / (sd[a] - sd[b]);
    V3 x = p.v[a] + ta * (p.v[b] - p.v[a]);
    int id = (int)nvtx.size();
    nvtx.push_back(x);
    cuts.push_back({key, id});
    return id;
  };
  std::vector<std::vector<int>> nf;
  std::vector<Tag> ntag;
  std::vector<std::pair<int, int>> cap;  // directed cap edges (from, to)
  for (size_t fi = 0; fi < p.f.size(); ++fi) {
    const auto& L = p.f[fi];
    const int m = (int)L.size();
    std::vector<int> out;
    int exitv = -1, entryv = -1;
    for (int k = 0; k < m; ++k) {
      int a = L[k], b = L[(k + 1) % m];
      bool ain = sd[a] <= 0, bin = sd[b] <= 0;
      if (ain) out.push_back(remap[a]);
      if (ain && !bin) {
        exitv = cut_vertex(a, b);
        out.push_back(exitv);
      } else if (!ain && bin) {
        entryv = cut_vertex(a, b);
        out.push_back(entryv);
      }
    }
    if (out.size() >= 3) {
      nf.push_back(out);
      ntag.push_back(p.tag[fi]);
    }
    // the face loop runs ... exit -> entry ... along the plane; the cap,
    // seen from outside along +n, runs entry -> exit
    if (exitv >= 0 && entryv >= 0 && exitv != entryv) cap.push_back({entryv, exitv});
  }
  if (cap.size() >= 3) {
    std::vector<int> loop;
    loop.push_back(cap[0].first);
    int cur = cap[0].second;
    size_t guard = 0;
    while (cur != loop[0] && guard++ < cap.size() + 2) {
      loop.push_back(cur);
      int nxt = -1;
      for (auto& e : cap)
        if (e.first == cur) {
          nxt = e.second;
          break;
        }
      if (nxt < 0) break;
      cur = nxt;
    }
    if (loop.size() >= 3) {
      nf.push_back(loop);
      ntag.push_back(t);
    }
  }
  // drop unreferenced vertices is unnecessary: all kept vertices lie on faces
  p.v.swap(nvtx);
  p.f.swap(nf);
  p.tag.swap(ntag);
  return true;
}

struct FaceOut {
  int32_t i, j;
  int8_t s[3];
  double area;
  V3 normal, centroid;
};

struct CellOut {
  double volume;
  V3 centroid;
};

struct Offset {
  int dx, dy, dz;
  double dist;
};

}  // namespace

struct VorMesh {
  int64_t n_cells = 0;
  std::vector<CellOut> cells;
  std::vector<FaceOut> faces;
  std::vector<int64_t> ptr;
  std::vector<int32_t> idx;
};

extern "C" {

// Builds the periodic Voronoi mesh of generators pts[N][3] that lie in the
// box [0,Lx)x[0,Ly)x[0,Lz) and were made from an nx*ny*nz lattice (point
// index = (ix*ny + iy)*nz + iz) with every coordinate displaced from its
// lattice site ((ix+0.5)Lx/nx, ...) by at most jit[d] (absolute units).
// Returns an opaque handle or NULL on bad arguments.
void* vor_build_lattice(const double* pts, int nx, int ny, int nz, const double* box,
                        const double* jit, int n_threads) {
  if (!pts || nx < 1 || ny < 1 || nz < 1 || !box || !jit) return nullptr;
  const int64_t N = (int64_t)nx * ny * nz;
  const V3 L = {box[0], box[1], box[2]};
  const V3 h = {L.x / nx, L.y / ny, L.z / nz};
  const V3 J = {jit[0], jit[1], jit[2]};
  const double jn = std::sqrt(dot(J, J));
  const double hn = std::sqrt(dot(h, h));
  // any point of a cell lies within 0.5|h| + |J| of its generator
  const double rmax_bound = 0.5 * hn + jn;
  // candidate offsets: lattice distance < 2*rmax_bound + 2|J|
  const double reach = 2.0 * rmax_bound + 2.0 * jn;
  int R[3] = {(int)std::ceil(reach / h.x), (int)std::ceil(reach / h.y),
              (int)std::ceil(reach / h.z)};
  std::vector<Offset> offs;
  for (int dx = -R[0]; dx <= R[0]; ++dx)
    for (int dy = -R[1]; dy <= R[1]; ++dy)
      for (int dz = -R[2]; dz <= R[2]; ++dz) {
        if (!dx && !dy && !dz) continue;
        double dd = std::sqrt((dx * h.x) * (dx * h.x) + (dy * h.y) * (dy * h.y) +
                              (dz * h.z) * (dz * h.z));
        if (dd - 2.0 * jn < reach) offs.push_back({dx, dy, dz, dd});
      }
  std::sort(offs.begin(), offs.end(), [](const Offset& a, const Offset& b) {
    if (a.dist != b.dist) return a.dist < b.dist;
    if (a.dx != b.dx) return a.dx < b.dx;
    if (a.dy != b.dy) return a.dy < b.dy;
    return a.dz < b.dz;
  });

  VorMesh* M = new VorMesh();
  M->n_cells = N;
  M->cells.resize(N);
  if (n_threads < 1) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  std::vector<std::vector<FaceOut>> tf(n_threads);
  std::atomic<int64_t> next(0);
  const int64_t chunk = 256;
  std::vector<std::vector<std::pair<int64_t, int64_t>>> tranges(n_threads);

  auto worker = [&](int tid) {
    Poly P;
    std::vector<double> sd;
    std::vector<int> remap;
    for (;;) {
      int64_t c0 = next.fetch_add(chunk);
      if (c0 >= N) break;
      int64_t c1 = std::min(N, c0 + chunk);
      tranges[tid].push_back({c0, (int64_t)tf[tid].size()});
      for (int64_t c = c0; c < c1; ++c) {
        const int ix = (int)(c / ((int64_t)ny * nz));
        const int iy = (int)((c / nz) % ny);
        const int iz = (int)(c % nz);
        const V3 pc = {pts[3 * c], pts[3 * c + 1], pts[3 * c + 2]};
        make_box(P, pc, {rmax_bound * 1.01, rmax_bound * 1.01, rmax_bound * 1.01});
        double r2 = 0;
        for (auto& x : P.v) r2 = std::max(r2, dot(x - pc, x - pc));
        for (const Offset& o : offs) {
          // lower bound on |p_j - p_c| for this offset; stop when it cannot cut
          if (o.dist - 2.0 * jn > 2.0 * std::sqrt(r2) * (1 + 1e-12)) break;
          int jx = ix + o.dx, jy = iy + o.dy, jz = iz + o.dz;
          int sx = (int)std::floor((double)jx / nx), sy = (int)std::floor((double)jy / ny),
              sz = (int)std::floor((double)jz / nz);
          jx -= sx * nx;
          jy -= sy * ny;
          jz -= sz * nz;
          const int64_t j = ((int64_t)jx * ny + jy) * nz + jz;
          const V3 pj = {pts[3 * j] + sx * L.x, pts[3 * j + 1] + sy * L.y,
                         pts[3 * j + 2] + sz * L.z};
          const V3 dvec = pj - pc;
          const double dl = std::sqrt(dot(dvec, dvec));
          if (dl > 2.0 * std::sqrt(r2) * (1 + 1e-12)) continue;
          const V3 n = (1.0 / dl) * dvec;
          const V3 mid = pc + 0.5 * dvec;
          Tag t{(int32_t)j, {(int8_t)sx, (int8_t)sy, (int8_t)sz}};
          if (clip(P, n, dot(n, mid), t, sd, remap)) {
            r2 = 0;
            for (auto& x : P.v) r2 = std::max(r2, dot(x - pc, x - pc));
          }
        }
        // geometry of the finished cell
        double vol = 0;
        V3 cen = {0, 0, 0};
        for (size_t fi = 0; fi < P.f.size(); ++fi) {
          const auto& Lp = P.f[fi];
          V3 av = {0, 0, 0}, fc = {0, 0, 0};
          double asum = 0;
          const V3 v0 = P.v[Lp[0]];
          for (size_t k = 1; k + 1 < Lp.size(); ++k) {
            V3 a = P.v[Lp[k]] - v0, b = P.v[Lp[k + 1]] - v0;
            V3 cr = cross(a, b);
            double ta = 0.5 * std::sqrt(dot(cr, cr));
            av = av + 0.5 * cr;
            V3 tc = (1.0 / 3.0) * (v0 + P.v[Lp[k]] + P.v[Lp[k + 1]]);
            fc = fc + ta * tc;
            asum += ta;
          }
          if (asum <= 0) continue;
          fc = (1.0 / asum) * fc;
          const Tag& t = P.tag[fi];
          if (t.j < 0) continue;  // box wall survived: impossible for valid inputs
          V3 pj = {pts[3 * t.j] + t.s[0] * L.x, pts[3 * t.j + 1] + t.s[1] * L.y,
                   pts[3 * t.j + 2] + t.s[2] * L.z};
          V3 dvec = pj - pc;
          V3 n = (1.0 / std::sqrt(dot(dvec, dvec))) * dvec;
          double area = dot(av, n);
          double pyr = area * dot(fc - pc, n) / 3.0;
          vol += pyr;
          cen = cen + pyr * (pc + 0.75 * (fc - pc));
          bool own = (t.j > c) ||
                     (t.j == c && (t.s[0] > 0 || (t.s[0] == 0 && (t.s[1] > 0 ||
                                                                (t.s[1] == 0 && t.s[2] > 0)))));
          if (own) {
            FaceOut fo;
            fo.i = (int32_t)c;
            fo.j = t.j;
            std::memcpy(fo.s, t.s, 3);
            fo.area = area;
            fo.normal = n;
            fo.centroid = fc;
            tf[tid].push_back(fo);
          }
        }
        M->cells[c].volume = vol;
        M->cells[c].centroid = (1.0 / vol) * cen;
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t) th.emplace_back(worker, t);
  for (auto& t : th) t.join();

  // gather faces in cell order (chunks were claimed in increasing order per
  // thread; merge all chunks by their first cell)
  struct Chunk {
    int64_t c0;
    int tid;
    int64_t begin, end;
  };
  std::vector<Chunk> chunks;
  for (int t = 0; t < n_threads; ++t)
    for (size_t k = 0; k < tranges[t].size(); ++k) {
      int64_t e = (k + 1 < tranges[t].size()) ? tranges[t][k + 1].second
                                              : (int64_t)tf[t].size();
      chunks.push_back({tranges[t][k].first, t, tranges[t][k].second, e});
    }
  std::sort(chunks.begin(), chunks.end(),
            [](const Chunk& a, const Chunk& b) { return a.c0 < b.c0; });
  size_t total = 0;
  for (auto& ch : chunks) total += ch.end - ch.begin;
  M->faces.reserve(total);
  for (auto& ch : chunks)
    for (int64_t k = ch.begin; k < ch.end; ++k) M->faces.push_back(tf[ch.tid][k]);
  tf.clear();
  // CSR: each face once in the list of i (as f) and once in that of j (as -(f+1))
  M->ptr.assign(N + 1, 0);
  for (auto& f : M->faces) {
    M->ptr[f.i + 1]++;
    M->ptr[f.j + 1]++;
  }
  for (int64_t c = 0; c < N; ++c) M->ptr[c + 1] += M->ptr[c];
  M->idx.resize(M->ptr[N]);
  std::vector<int64_t> fill(M->ptr.begin(), M->ptr.end() - 1);
  for (size_t f = 0; f < M->faces.size(); ++f) {
    M->idx[fill[M->faces[f].i]++] = (int32_t)f;
    M->idx[fill[M->faces[f].j]++] = -(int32_t)f - 1;
  }
  return M;
}

void vor_sizes(void* h, int64_t* n_cells, int64_t* n_faces, int64_t* nnz) {
  VorMesh* M = (VorMesh*)h;
  *n_cells = M->n_cells;
  *n_faces = (int64_t)M->faces.size();
  *nnz = (int64_t)M->idx.size();
}

// Copies the mesh out: volume[N], centroid[N][3], face_cells[Nf][2],
// face_shift[Nf][3], face_area[Nf], face_normal[Nf][3], face_centroid[Nf][3],
// cell_face_ptr[N+1], cell_face_idx[nnz].
void vor_fetch(void* h, double* volume, double* centroid, int32_t* face_cells,
               int8_t* face_shift, double* face_area, double* face_normal,
               double* face_centroid, int64_t* ptr, int32_t* idx) {
  VorMesh* M = (VorMesh*)h;
  for (int64_t c = 0; c < M->n_cells; ++c) {
    volume[c] = M->cells[c].volume;
    centroid[3 * c] = M->cells[c].centroid.x;
    centroid[3 * c + 1] = M->cells[c].centroid.y;
    centroid[3 * c + 2] = M->cells[c].centroid.z;
  }
  for (size_t f = 0; f < M->faces.size(); ++f) {
    const FaceOut& F = M->faces[f];
    face_cells[2 * f] = F.i;
    face_cells[2 * f + 1] = F.j;
    face_shift[3 * f] = F.s[0];
    face_shift[3 * f + 1] = F.s[1];
    face_shift[3 * f + 2] = F.s[2];
    face_area[f] = F.area;
    face_normal[3 * f] = F.normal.x;
    face_normal[3 * f + 1] = F.normal.y;
    face_normal[3 * f + 2] = F.normal.z;
    face_centroid[3 * f] = F.centroid.x;
    face_centroid[3 * f + 1] = F.centroid.y;
    face_centroid[3 * f + 2] = F.centroid.z;
  }
  std::memcpy(ptr, M->ptr.data(), sizeof(int64_t) * M->ptr.size());
  std::memcpy(idx, M->idx.data(), sizeof(int32_t) * M->idx.size());
}

void vor_free(void* h) { delete (VorMesh*)h; }

}  // extern "C"
