// Internal declarations of the GB300 radiation library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rt.h"

namespace rt {

constexpr double kPi = 3.14159265358979323846;

// Directed face slot of one cell, in the cell's outward orientation.  The
// volume flux coefficient of angle a through the face is
//   u_a = cbar A_f (n_a . n_f) - A_f (w_f . n_f)       (n_f outward).
// Float states store s = cbar A_f n_f and w = A_f w_f . n_f and evaluate
// n_a . s - w with FMAs.  Double states store n_f and cbar A_f and evaluate
// cbar A_f ((n_ax n_fx + n_ay n_fy) + n_az n_fz) - W without contraction, in
// the same order as a plain evaluation of the formula: near-tangent faces
// make this a cancelling dot product whose last bits decide the flux of a
// faint intensity next to a bright one.  The slot on the other side of a face
// holds the exact negatives (W in a separate array for double states).
struct alignas(16) SlotF {
  float sx, sy, sz, w;
};
struct alignas(32) SlotD {
  double nx, ny, nz, ca;
};
template <typename R> struct SlotOf;
template <> struct SlotOf<float> { using type = SlotF; };
template <> struct SlotOf<double> { using type = SlotD; };

// Status bits latched by the step kernels.
enum : unsigned {
  ST_NONCONV = 1u,
  ST_NONFINITE = 2u,
  ST_CFL = 4u,  // a cell's current volume is below dt max_a sum_f max(u, 0) (gcl states)
};

// The step kernel works on blocks of CPB consecutive (internal) cells.
constexpr int CPB = 32;
// Face slots of one block of CPB cells that the float QuadMap kernel stages
// in shared memory at most; meshes with more take the PairMap kernel.
constexpr int STAGE_SLOTS = 1024;

// Per-cell constant gas data: rho, the absorption / scattering coefficients
// rho kappa_P, rho kappa_J, rho kappa_s, 1/rho and
// rho c_v = rho r_gas / (gamma - 1) in double, and float copies of the
// coefficients and rho c_v for the float states' temperature solve.
struct alignas(64) GasStatic {
  double rho, rkP, rkJ, rkS, inv_rho, rcv;
  float frkP, frkJ, frkS, frcv;
};
// Per-cell evolving gas data (double): e, m.
struct alignas(32) GasDyn {
  double e, mx, my, mz;
};

// Gas dynamics (rt_hydro.cu): one record per face (caller face order) and
// one per directed slot (internal slot order).
struct HydroFace {
  int32_t i, j;        // internal cells: first (left) and second (right)
  double area;
  double n[3];         // unit normal, i -> j
  double oi[3], oj[3]; // face centroid minus the centroid of i and of j' (j's image across the face)
};
struct HydroSlot {
  double own[3], nbr[3];  // face centroid minus the cell's / the neighbour image's centroid
  double area;
  double sign;            // +1: the cell is the face's first cell, -1: its second
  int64_t face;           // caller face index (into the face fluxes)
  double wr[3];           // least-squares weight A_f / |r|^2 times r = own - nbr (set on the device)
};

template <typename R> struct StepArgs {
  int64_t n_cells;
  int32_t n_angles, half;
  int32_t row;              // reals between intensity rows (I_in, I_out, I0)
  const int64_t *ptr;       // [N+1] slot range per internal cell
  const int32_t *nbr;       // [nnz] internal neighbour index
  const typename SlotOf<R>::type *slot;  // [nnz]
  const SlotF *slot_nb;     // [nnz] float static meshes: (s, neighbour index bits)
  const double *uface;      // [nnz][A/2] double states: flux coefficient of pair p through slot k
  const R *inv_vol;         // [N]
  const double *wface;      // [nnz] A_f w_f . n_f of double slots (moving meshes)
  const GasStatic *gs;      // [N]
  GasDyn *gd;               // [N]
  const uint8_t *kind;      // [N]
  const double2 *aux;       // [N] (tau or emit_rate, I_src)
  const int32_t *bc_row;    // [N]
  const R *I0;              // [rows][A]
  double *ext;              // [N][4]
  const R *dir;             // [A][4] (x, y, z, 0), caller angle order
  const R *wt2;             // [A/2][2] (w_p, w_{p+A/2})
  const R *I_in;            // [N][A]
  R *I_out;                 // [N][A]
  R *cellv;                 // [N][4] (v_x, v_y, v_z, e - rho v^2 / 2)
  double dt, cbar, c, a_rad, rcv;  // rcv = r_gas / (gamma - 1)
  double k_dcr, k_alpha, k_g, k_fe, k_fm;  // dt cbar, dt c a, dt c 4 pi, 4 pi c/cbar, 4 pi/cbar
  R dt_r, dt_cbar_r, inv_c_r;
  float k_dcr_f, k_alpha_f, k_g_f, a_rad_4pi_f;  // float copies for the float quartic
  int32_t newton_max_iter;
  int32_t float_quartic;    // float states: 1 solves the quartic in float in every lane
  int32_t src_only;         // 1: I_in holds I* already (no transport)
  int32_t commit;           // 0: the gas update is discarded (van Leer stage 1)
  int32_t boost;            // 1: Gamma = gamma (1 -+ v.n/c) with the Lorentz factor gamma
  // geometric conservation law (NULL: fixed volumes): per-cell sum_f A w . n,
  // per-cell max_a sum_f max(u, 0), the current volumes and their inverses
  const double *gcl_rate;
  const float *gcl_kv;
  double gcl_kv_unit;       // gcl_kv times this is max_a sum_f max(u, 0)
  double *volume;
  R *inv_vol_w;
  // temperature-dependent opacities (0, 0: constant): kappa_P (T/T_ref)^beta_P
  // at T^{n+1} in the temperature solve, kappa_J (T/T_ref)^beta_J refreshed
  // from T^{n+1} in the gas phase for the next step (rkJ0: rho kappa_J at T_ref)
  double beta_P, beta_J, T_ref, tref_mbP;  // tref_mbP = T_ref^-beta_P
  float beta_P_f, T_ref_f, tref_mbP_f;
  const double *rkJ0;
  GasStatic *gs_w;
  unsigned *status;
  unsigned long long *bad_cell;
};

}  // namespace rt

// Internal intensity rows.  Pair p < A/2 couples angle p with its antipode
// p + A/2.  Positions q >= quad_end store the pairs side by side (2p + s
// holds angle p + s A/2).  Positions q < quad_end (float states with A a
// multiple of 16; quad_end = 32 floor(A/32), else 0) group two pairs per
// four positions: 4Q, 4Q+1, 4Q+2, 4Q+3 hold angles 2Q, 2Q+1, 2Q + A/2,
// 2Q+1 + A/2, so one 16-byte access gives a thread both pairs with the
// angles of one hemisphere side by side.
__host__ __device__ inline int angle_of_position(int q, int half, int quad_end) {
  if (q < quad_end) return 2 * (q >> 2) + (q & 1) + ((q & 2) ? half : 0);
  return (q & 1) ? (q >> 1) + half : (q >> 1);
}
__host__ __device__ inline int position_of_angle(int a, int half, int quad_end) {
  const int p = a < half ? a : a - half, s = a < half ? 0 : 1;
  if (2 * p < quad_end) return 4 * (p >> 1) + (p & 1) + 2 * s;
  return 2 * p + s;
}

// Opaque state behind the C ABI.
struct rt_state {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = RT_FP64;
  size_t rsize = 8;  // bytes per real of the state precision
  int64_t n_cells = 0, n_faces = 0, nnz = 0;
  int32_t n_angles = 0;
  rt_params params{};
  double dt_cfl = 0, dt_max = 0;
  bool gas_set = false;
  bool moving = false;  // some face has a non-zero velocity
  int64_t max_block_slots = 0;  // max over blocks of CPB cells of their face slots
  int quad_end = 0;  // internal row layout (see angle_of_position)
  int32_t row_stride = 0;  // reals between internal rows of d_I[0], d_I[1], d_I0 (>= n_angles)
  int64_t n_rows = 0;
  std::string err;
  int64_t launches = 0;
  // captured step sequences of multi-step launches (rt_run / rt_launch), one
  // per buffer parity: replayed only for the dt and the generation they were
  // captured at (gen counts the rt_set_* calls, which may change arguments)
  bool plain_launches = false;
  uint64_t gen = 1;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaStream_t cap_stream = nullptr;  // the stream graphs are captured on
  // pipelined host I/O (rt_step_io): the copy-engine streams, the device
  // staging rows of the host copies (caller order), and the events that
  // order them: ev_h2d the rows landed, ev_pin the staged input consumed,
  // ev_pout the result staged, ev_d2h the result copied out
  cudaStream_t io_in = nullptr, io_out = nullptr;
  void *d_io_in = nullptr, *d_io_out = nullptr;
  cudaEvent_t ev_h2d = nullptr, ev_pin = nullptr, ev_pout = nullptr, ev_d2h = nullptr;
  double graph_dt[2] = {0.0, 0.0};
  uint64_t graph_gen[2] = {0, 0};
  int64_t graph_launches[2] = {0, 0};
  size_t device_bytes = 0;
  // power of two by which the positivity screen's float slots are scaled
  // (double states: brings cbar A near 1; float states: 1); the per-cell
  // factors in d_gcl_kv are in those scaled units
  double screen_scale = 1.0;

  // host copies needed for I/O
  std::vector<int64_t> cell_of;  // internal -> caller
  std::vector<double> volume;    // caller order

  // device buffers
  int64_t *d_ptr = nullptr;
  int32_t *d_nbr = nullptr;

  void *d_slot = nullptr;
  rt::SlotF *d_slot_nb = nullptr;  // float, static mesh: slot with the neighbour in w
  double *d_uface = nullptr;  // double: [nnz][A/2] flux coefficients, built once (build_uface)
  // van Leer integrator: reconstruction geometry ([nnz][8] and [N][8] reals
  // of the state precision, see build_recon), stage-1 intensities [N][RS]
  // and their limited gradients [3][N][RS] (x, y, z rows in the row layout)
  int integrator = RT_FIRST_ORDER;
  void *d_recon = nullptr, *d_lsq = nullptr, *d_Ihalf = nullptr, *d_grad = nullptr;
  double *d_wface = nullptr;  // double states: per-slot A w . n
  // geometric conservation law: per-cell volume rate sum_f A w . n (double,
  // internal order) and max_a sum_f max(u, 0) (float); NULL when off
  double *d_gcl_rate = nullptr;
  float *d_gcl_kv = nullptr;
  // temperature-dependent kappa_J: rho kappa_J at T_ref (internal order)
  double *d_rkJ0 = nullptr;
  // frequency groups (1: grey): the kernels see n_groups copies of the base
  // angle set as one set in the internal angle order (first halves of all
  // groups, then the second halves); col_of_angle maps an internal angle to
  // its caller column j A + a; d_kapg [N][n_groups][3] rho kappa_P, J, s
  int n_groups = 1;
  std::vector<double> group_w;
  std::vector<int32_t> col_of_angle;
  double *d_kapg = nullptr;
  float *d_kapgf = nullptr;  // [N][n_groups][4] float copies (rho kappa_P, J, s, 0)
  void *d_inv_vol = nullptr;
  int64_t *d_cell_of = nullptr;  // internal -> caller
  double *d_volume = nullptr;    // internal order
  rt::GasStatic *d_gs = nullptr;
  rt::GasDyn *d_gd = nullptr;
  uint8_t *d_kind = nullptr;
  double2 *d_aux = nullptr;
  int32_t *d_bc_row = nullptr;
  void *d_I0 = nullptr;
  double *d_ext = nullptr;
  void *d_cellv = nullptr;  // [N][4] in the state precision
  void *d_dir = nullptr;       // [A][4], caller angle order
  void *d_wt = nullptr;        // [A/2][2] weights of the pairs (p, p + A/2)
  double *d_dir64 = nullptr;   // [A][3] double, internal angle order
  double *d_wt64 = nullptr;    // [A], internal angle order
  int32_t *d_angle_of = nullptr;  // internal angle position -> caller angle
  int32_t *d_pos_of = nullptr;    // caller angle -> internal angle position
  void *d_I[2] = {nullptr, nullptr};
  int cur = 0;
  unsigned *d_status = nullptr;
  unsigned long long *d_bad = nullptr;
  void *d_adj[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double *d_adj_ws = nullptr;     // [25 N] adjoint per-cell records (internal order)
  double *d_adj_stage = nullptr;  // [10 N] host-path staging of per-cell vectors
  // gas dynamics (params.hydro): face and slot records, work area
  rt::HydroFace *d_hface = nullptr;
  rt::HydroSlot *d_hslot = nullptr;
  double *d_hlsq = nullptr;  // [N][10] cofactors and determinant of each cell's normal matrix
  double *d_hwork = nullptr;
  double *d_scratch = nullptr;  // reduction partials
  size_t scratch_len = 0;
  double *d_out16 = nullptr;
};

namespace rt {

// kernel launchers (rt_step.cu)
cudaError_t launch_step(rt_state *s, double dt);
// One launch of the step kernel with explicit rows: `in` -> `out`; src_only:
// `in` already holds the transported I* (the source step only); commit:
// write the gas update (else only the status bits).
struct StepIO {
  const void *in;
  void *out;
  bool src_only, commit;
};
cudaError_t launch_step_io(rt_state *s, double dt, const StepIO &io);
// Transport only (rt_transport.cu), rows `in` -> `out` (stride row_stride):
// adjoint = false: I* = I - dt/V sum_f u I_up; adjoint = true: the
// transposed operator, from rows L = dt/V lambda to M^T lambda.
cudaError_t launch_transport(rt_state *s, double dt, const void *in, void *out, bool adjoint);
// The coupled source step of frequency groups (rt_groups.cu), in place on
// the transported rows I* (stride row_stride).
cudaError_t launch_group_source(rt_state *s, double dt, void *Is);
// one step of a grouped state: In = I^n rows, Out = I^{n+1} rows
cudaError_t launch_group_step(rt_state *s, double dt, const void *In, void *Out);
// The van Leer step (rt_recon.cu); leaves I^{n+1} in d_I[cur ^ 1].
cudaError_t launch_step_vl(rt_state *s, double dt);
// Double states: fills d_uface (allocates it on first use).
cudaError_t build_uface(rt_state *s);

// A CUDA driver function by name (through the runtime's entry-point query,
// so the library does not link the driver library itself), or NULL.
void *driver_fn(const char *name);
// Identifier of the current context (unique for the process), 0 if unknown.
unsigned long long current_context_id();

// gas dynamics (rt_hydro.cu)
int hydro_setup(rt_state *s, const rt_mesh_desc *m);
cudaError_t launch_hydro_step(rt_state *s, double dt, int order);
cudaError_t launch_hydro_dt(rt_state *s, double cfl, double *dt);
cudaError_t launch_density_out(rt_state *s, double *rho);
double *hydro_kmass(rt_state *s);  // [N][3] opacities per unit mass, internal order

// auxiliary kernels (rt_aux.cu)
// caller order <-> internal order; the internal rows are `stride` reals apart
cudaError_t launch_permute_in(rt_state *s, const void *src, void *dst, int stride);
cudaError_t launch_permute_out(rt_state *s, const void *src, void *dst, int stride);
// the same with the caller's rows in page-locked host memory (src / dst: the
// device-side address of that memory): every caller row is read or written
// whole and in order, so the host link sees full lines
cudaError_t launch_permute_in_host(rt_state *s, const void *src, void *dst, int stride);
cudaError_t launch_permute_out_host(rt_state *s, const void *src, void *dst, int stride);
// kcell (may be NULL): per cell max_a sum_f max(u, 0), float
cudaError_t launch_positivity(rt_state *s, const SlotF *fslot, double *d_kmax, float *kcell);
// inv_vol = 1 / volume (state precision) after the volumes changed
cudaError_t launch_inv_vol(rt_state *s);
// rho kappa_J(T) = rkJ0 (T / T_ref)^beta_J of every cell from its gas state
cudaError_t launch_opacity_refresh(rt_state *s);
cudaError_t launch_moments(rt_state *s, double *E, double *F, double *P);
cudaError_t launch_totals(rt_state *s, double *d_out16);
// the same sums with the per-block partials in `partial` (room for
// ceil(n_cells / cpb) x 12 doubles), blocks of cpb >= 1 cells; rt_totals
// takes cpb = totals_block_cells
constexpr int64_t totals_block_cells = 64;
cudaError_t launch_totals_with(rt_state *s, double *partial, int64_t cpb, double *d_out16);
cudaError_t launch_gas_out(rt_state *s, double *e, double *m, double *ext);
// caller-order device (e, m) into the internal gas records
cudaError_t launch_gas_in(rt_state *s, const double *e, const double *m);
cudaError_t launch_cellv(rt_state *s);

// adjoint (rt_adjoint.cu): device pointers, caller order
cudaError_t adjoint_step(rt_state *s, double dt, const void *I, const double *e, const double *m,
                         const void *lI1, const double *le1, const double *lm1, void *lI,
                         double *le, double *lm, double *gP, double *gJ);

}  // namespace rt
