/*
 * rt.h -- C ABI of the GB300 reduced-speed-of-light radiative-transfer step
 * on an unstructured (Voronoi) mesh.
 *
 * The method is that of Chang, Davis & Jiang, "Time dependent radiation
 * hydrodynamics on a moving mesh": discrete-ordinate intensities I(cell,
 * angle) are transported across the mesh faces by an upwind finite-volume
 * flux (Sec. 2.2) and then updated by an implicit, per-cell source step in
 * the fluid's comoving frame that solves a quartic for the gas temperature
 * and returns the energy and momentum exchange to the gas (Sec. 2.3).
 * Boundary cells relax to a prescribed field (Sec. 2.4) and emitter cells
 * relax to a source intensity (Sec. 2.5).
 *
 * Conventions shared by every call
 *   - Plain C types only.  Arrays are row-major and, unless a call takes an
 *     on_device flag that is set, HOST pointers.  Device pointers passed
 *     with on_device = 1 must be valid on the state's device and are used
 *     on the state's stream only for the duration of the call.
 *   - Cells and angles are numbered as the caller numbers them.  The
 *     library may store cells in another order internally; every input and
 *     output is converted.
 *   - Units: intensities are energy density per steradian, so an isotropic
 *     equilibrium field is I = a_rad T^4 / (4 pi); E_r = 4 pi sum_a w_a I_a,
 *     F_r = 4 pi c sum_a w_a n_a I_a, P_r = 4 pi sum_a w_a n_a n_a I_a
 *     (Sec. 2.1 moments with sum_a w_a = 1).  The gas has e = total energy
 *     density, m = momentum density, ideal-gas temperature
 *     T = (gamma - 1)(e - |m|^2 / (2 rho)) / (rho r_gas).
 *   - Every call returns an rt_status.  On failure rt_last_error() gives a
 *     one-line description.  Per-cell failures inside a step (Newton not
 *     converged, non-finite values) are latched on the device and returned
 *     by the call that synchronises (rt_step / rt_run / rt_totals / rt_sync).
 *   - The library allocates its device memory in rt_create and frees it in
 *     rt_destroy.  It keeps no pointer to caller memory after a call returns.
 *     Besides the two intensity buffers (N A reals each) and the mesh, an
 *     RT_FP64 state holds a table of the flux coefficients, A/2 doubles per
 *     directed face (8 A/2 x 2 N_faces bytes), so that its steps do not
 *     recompute them.
 */
#ifndef RT_GB300_H
#define RT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_state rt_state;

typedef enum {
  RT_OK = 0,
  RT_ERR_ARG = -1,       /* bad argument (null pointer, size, flag)            */
  RT_ERR_MESH = -2,      /* mesh fails validation (index range, open cell)      */
  RT_ERR_CUDA = -3,      /* CUDA runtime error                                  */
  RT_ERR_OOM = -4,       /* device allocation failed                            */
  RT_ERR_CFL = -5,       /* dt above the upwind positivity limit                */
  RT_ERR_NONCONV = -6,   /* temperature Newton iteration did not converge       */
  RT_ERR_NONFINITE = -7, /* non-finite intensity or temperature produced        */
  RT_ERR_STATE = -8      /* call out of order (e.g. step before rt_set_gas)     */
} rt_status;

typedef enum {
  RT_FP64 = 0, /* every quantity in double precision                          */
  RT_FP32 = 1  /* intensities, face geometry and the transport sweep in float;
                  the temperature quartic, the gas energy/momentum exchange
                  and the conservation sums in double                         */
} rt_precision;

typedef enum {
  RT_CELL_INTERIOR = 0, /* transport + implicit gas coupling (Sec. 2.3)       */
  RT_CELL_BOUNDARY = 1, /* I -> I - (I - I0) min(dt/tau, 1) (Sec. 2.4)         */
  RT_CELL_EMITTER = 2   /* comoving I~ relaxes to I_src at rate cbar*emit_rate
                           (Sec. 2.5)                                          */
} rt_cell_kind;

/* Mesh and angle set (Sec. 2: Voronoi cells i with volume V_i, faces with
 * area A_ij, unit normal n_ij pointing from i to j; Sec. 2.2: face velocity
 * w_ij).  All pointers are host pointers, copied by rt_create.
 *   face_cells[f] = (i, j): a face is listed once; i == j is allowed (a cell
 *     meeting its own periodic image).
 *   cell_face_ptr/cell_face_idx: CSR over cells; entry f >= 0 means the cell
 *     is face f's first cell (outward normal +n_f), entry -(f+1) means it is
 *     the second cell (outward normal -n_f).  The order of a cell's entries is
 *     the order in which its face fluxes are summed.
 *   angle_dir[A][3] unit directions, angle_w[A] weights with sum 1.  The set
 *     must be centrally symmetric in the order angle_dir[a + A/2] =
 *     -angle_dir[a] (A even); rt_create rejects it otherwise.
 *   face_w may be NULL (static mesh).  cell_centroid and face_centroid are
 *     used for the locality ordering only and may be NULL.
 *   face_offset[f] = (x_f - x_i, x_f - x_j'): the face centroid minus each
 *     cell's centroid, j' being the image of j that meets i across the face
 *     (on a periodic mesh the two cells' centroids may lie in different
 *     periodic frames).  Required when params->integrator = RT_VAN_LEER (the
 *     linear reconstruction of Sec. 2.2), ignored and may be NULL otherwise.
 *   n_groups > 1: frequency groups (Sec. 2.3) that share the angle set and
 *     couple only through the gas temperature.  Group j has weight
 *     group_w[j] > 0 (sum 1); intensities are [N][n_groups][A] (every
 *     intensity argument then holds n_groups * A values per cell, I0 rows
 *     too), rt_set_gas takes kappa_P, kappa_J, kappa_s as [N][n_groups], and
 *     rt_moments / rt_totals report the group-weighted sums.  Needs
 *     n_groups * A <= 128, RT_FIRST_ORDER, boost = 0, gcl = 0 and constant
 *     opacities; rt_adjoint_step refuses it.  A step is then two launches: the
 *     transport of all groups' intensities and the coupled source step. */
typedef struct {
  int64_t n_cells;
  int64_t n_faces;
  int32_t n_angles;
  int32_t n_groups;            /* frequency groups; 0 or 1: grey */
  const double *cell_volume;   /* [N]        */
  const double *cell_centroid; /* [N][3]     */
  const int32_t *face_cells;   /* [Nf][2]    */
  const double *face_area;     /* [Nf]       */
  const double *face_normal;   /* [Nf][3]    */
  const double *face_centroid; /* [Nf][3]    */
  const double *face_w;        /* [Nf][3]    */
  const int64_t *cell_face_ptr;/* [N+1]      */
  const int32_t *cell_face_idx;/* [nnz]      */
  const double *angle_dir;     /* [A][3]     */
  const double *angle_w;       /* [A]        */
  const double *face_offset;   /* [Nf][2][3] */
  const double *group_w;       /* [n_groups], n_groups > 1 only */
} rt_mesh_desc;

/* Time integration of the transport (Sec. 2, integration steps).
 *   RT_FIRST_ORDER: piecewise-constant upwind transport over dt, then the
 *     implicit source over dt.
 *   RT_VAN_LEER: the paper's van Leer half step.  Stage 1 takes the first-
 *     order step over dt/2 (its gas update is discarded); stage 2 applies to
 *     I^n the fluxes of the stage-1 intensities reconstructed linearly at the
 *     face centres -- least-squares gradients over the face neighbours,
 *     limited (Barth-Jespersen) to the range of the cell and its neighbours --
 *     then the implicit source over dt from the gas at the start of the step.
 *     Second order in smooth regions, first order at extrema. */
typedef enum { RT_FIRST_ORDER = 0, RT_VAN_LEER = 1 } rt_integrator;

/* Physical constants and numerics (Sec. 2.1, 2.3.1).  cbar is the reduced
 * speed of light of the transport, c the true one (enters the gas coupling
 * and the moments).  r_gas = k_B / (mu m_p); c_v = r_gas / (gamma_gas - 1).
 * cfl scales the Courant step dt = cfl * min V^(1/3) / (cbar + |w|).
 * newton_max_iter <= 0 selects 64.  boost selects the frequency ratio of the
 * comoving transformation (Sec. 2.3), Gamma_a = gamma (1 - v . n_a / c):
 * 0 takes gamma = 1 (first order in v/c), 1 the Lorentz factor
 * gamma = (1 - v^2 / c^2)^(-1/2) of the cell's frame velocity (all orders;
 * every cell must then have |v| < c).  rt_adjoint_step reverses boost = 0
 * states only.
 * gcl = 1 lets the cell volumes follow the face velocities by the geometric
 * conservation law: every step takes V^{n+1} = V^n + dt sum_f A_f w_f . n_f
 * (faces in list order) and the conservative moving-cell transport
 * V^{n+1} I* = V^n I - dt sum_f u I_up, so a uniform field stays uniform on
 * any moving mesh.  The faces (areas, normals, w) stay the state's; the gas
 * density is not changed.  The upwind positivity limit then changes with the
 * volumes: rt_step checks dt against the creation limit on the host and every
 * cell against its current volume on the device (RT_ERR_CFL, latched like
 * the other per-cell failures).  rt_totals, rt_get_state and rt_set_state
 * use and keep the current volumes.  gcl = 1 needs RT_FIRST_ORDER;
 * rt_adjoint_step refuses gcl states.
 * beta_P, beta_J, T_ref: temperature-dependent opacities (Sec. 2.3 solves
 * the temperature equation by Newton-Raphson for them).  The cell's kappa_P
 * and kappa_J of rt_set_gas hold at T_ref; kappa_P(T) = kappa_P (T/T_ref)^beta_P
 * is taken at T^{n+1} inside the temperature solve (alpha T^(4 + beta_P) +
 * rho c_v T = g, beta_P >= -3), kappa_J(T) = kappa_J (T/T_ref)^beta_J at the
 * temperature at the start of each step.  0, 0: constant opacities (T_ref is
 * then unused; otherwise T_ref > 0).  rt_adjoint_step refuses beta != 0.
 * plain_launches = 0 (the default) lets rt_run / rt_launch replay a CUDA
 * graph of RT_GRAPH_STEPS steps captured on the state's stream (see rt_run);
 * 1 launches every kernel from the host.  Both give identical results.
 * float_quartic (RT_FP32 states only, ignored for RT_FP64): 0, the default,
 * solves the gas temperature equation of Eq. (com rad thermal disc) in
 * double -- its coefficients formed in double from the float angular sums,
 * Newton in double, one GPU lane per cell -- as the precision split of
 * RT_FP32 states says; 1 solves it in float in every lane of the cell (no
 * block barrier, faster; coefficients outside float range still take the
 * double solve), so the temperature carries float rounding.
 * hydro = 1 lets the state evolve the gas by the Euler equations as well
 * (rt_hydro_step, rt_radhydro_step: Sec. 2, radiation subcycled under a
 * hydro step); it needs face_offset, a static mesh (face_w NULL or zero),
 * n_groups 1, gcl 0 and constant opacities, and adds about 150 bytes per
 * face and 230 per cell of device memory. */
typedef struct {
  double cbar, c, a_rad, gamma_gas, r_gas, cfl;
  int32_t precision;       /* rt_precision */
  int32_t newton_max_iter;
  int32_t integrator;      /* rt_integrator */
  int32_t boost;           /* 0 or 1, see above */
  int32_t gcl;             /* 0 or 1, see above */
  int32_t plain_launches;  /* 0: multi-step calls replay captured graphs; 1: plain launches */
  double beta_P, beta_J, T_ref; /* see above */
  int32_t float_quartic;   /* RT_FP32 only: 0 temperature solve in double, 1 in float */
  int32_t hydro;           /* 1: the state also evolves the gas dynamics (rt_hydro_step) */
} rt_params;

/* Validates and copies the mesh to the device, orders cells for locality,
 * builds the per-cell directed face lists (bit-exact negated geometry on the
 * two sides of every face) and the upwind positivity bound.  stream is a
 * cudaStream_t (NULL = legacy default stream) on the current device; every
 * later call runs on it.  On success *out owns all device memory.
 * Errors: RT_ERR_ARG, RT_ERR_MESH (face index out of range, CSR not
 * consistent with face_cells, non-positive volume, open cell with
 * |sum_f A n| > 1e-9 sum_f A), RT_ERR_OOM, RT_ERR_CUDA. */
int rt_create(const rt_mesh_desc *mesh, const rt_params *params, void *stream,
              rt_state **out);

/* Gas state per cell (Sec. 2.3): rho, total energy density e, momentum
 * density m[N][3], Planck / mean / scattering opacities per unit mass.  The
 * frame velocity of a cell's source step is m / rho.  Host pointers, copied.
 * Resets the boundary / emitter tallies. */
int rt_set_gas(rt_state *s, const double *rho, const double *e, const double *m,
               const double *kappa_P, const double *kappa_J, const double *kappa_s);

/* Replaces only the evolving gas state -- total energy density e[N] and
 * momentum density m[N][3], caller order -- keeping rho, the opacities, the
 * cell kinds and the boundary / emitter tallies of the state (Sec. 2.3: the
 * quantities the source step updates).  For restoring a checkpoint (the
 * adjoint's recomputation) without the host round trip of rt_set_gas.
 * on_device = 1: e and m are device pointers on the state's device (their
 * values are not checked; a non-finite value surfaces as RT_ERR_NONFINITE in
 * the next step); 0: host pointers, checked finite (RT_ERR_ARG).  Needs a
 * prior rt_set_gas (RT_ERR_STATE). */
int rt_set_gas_energy(rt_state *s, const double *e, const double *m, int on_device);

/* Cell kinds (rt_cell_kind, [N]).  Boundary cells use tau[N] and the row
 * bc_row[N] of I0[n_rows][A]; emitter cells use emit_rate[N] (= rho kappa of
 * the source) and I_src[N].  kind == NULL makes every cell interior (the
 * other pointers may then be NULL).  Host pointers, copied. */
int rt_set_cells(rt_state *s, const uint8_t *kind, const double *tau, const double *emit_rate,
                 const double *I_src, const int32_t *bc_row, int64_t n_rows, const double *I0);

/* Intensities I[N][A] in the state's precision (float for RT_FP32, double
 * for RT_FP64), caller order.  on_device = 1: I is a device pointer. */
int rt_set_intensity(rt_state *s, const void *I, int on_device);
int rt_get_intensity(rt_state *s, void *I, int on_device);

/* Gas output: e[N], m[N][3] and the tallies ext[N][4] (energy and momentum
 * density handed to boundary and emitter reservoirs, positive = taken from
 * the radiation).  Any pointer may be NULL.  Double precision. */
int rt_get_gas(rt_state *s, double *e, double *m, double *ext, int on_device);

/* dt_cfl: the Courant step of rt_params.cfl; dt_max: the largest dt for
 * which every upwind update keeps a non-negative weight on its own cell,
 * 1 / max_{c,a} (1/V_c) sum_f max(u_fa, 0).  Either pointer may be NULL. */
int rt_dt_limits(rt_state *s, double *dt_cfl, double *dt_max);

/* One full step (Sec. 2.2 transport over dt, then the Sec. 2.3 source step
 * over dt): dt <= 0 selects dt_cfl.  Fails with RT_ERR_CFL if dt > dt_max.
 * Synchronises the stream and returns the first per-cell failure, if any
 * (the state then holds the partially failed step). */
int rt_step(rt_state *s, double dt, double *dt_used);

/* n_steps full steps with the same dt, launched back to back; synchronises
 * once at the end.  Unless rt_params.plain_launches is set, whole blocks of
 * RT_GRAPH_STEPS steps are replayed from a CUDA graph captured on the
 * state's stream (one launch of the graph instead of one per kernel; the
 * same kernels with the same arguments in the same order).  The graph is
 * captured (on a stream the state creates for that) at the first such call,
 * per dt and buffer parity, and captured again after any rt_set_* call.  No
 * graph is used while the caller is capturing the state's stream itself; the
 * steps are then launched one by one. */
#define RT_GRAPH_STEPS 16
int rt_run(rt_state *s, int32_t n_steps, double dt, double *dt_used);

/* Launches n_steps full steps without waiting for them; per-cell failures
 * are latched and returned by the next synchronising call (rt_sync,
 * rt_step, rt_run, rt_totals).  dt and the CFL check as for rt_step. */
int rt_launch(rt_state *s, int32_t n_steps, double dt, double *dt_used);

/* One full step whose intensities come from and go to page-locked host
 * memory, queued without waiting (a serving loop of rt_set_intensity,
 * rt_step, rt_get_intensity whose host copies overlap the GPU work): the
 * rows I_in[N][A] (caller order, state precision) replace the state's
 * intensities, one step runs (as rt_step: dt <= 0 selects dt_cfl,
 * RT_ERR_CFL if dt > dt_max), and the new rows are written to I_out[N][A].
 * The host copies run on the copy engines, on two streams of the state,
 * into and out of two device staging arrays that the device permutes then
 * read and write: a call's input copy overlaps the previous call's step and
 * result copy.  I_in and I_out must be page-locked in full (cudaHostAlloc /
 * cudaHostRegister; RT_ERR_ARG otherwise) and left alone until rt_sync (or
 * any call that returns the latched status) returns; an I_out must not be
 * the I_in of a call queued after it.  Per-cell failures latch as for
 * rt_launch.  The first call allocates the two staging arrays (the size of
 * the intensities each), kept until rt_destroy.  The results equal
 * rt_set_intensity, rt_step, rt_get_intensity bit for bit. */
int rt_step_io(rt_state *s, double dt, const void *I_in, void *I_out);

/* Lab-frame moments (Sec. 2.1 / Eqs. moments energy, moments flux) of the
 * current intensities, double precision, caller order: E[N], F[N][3],
 * P[N][6] (xx, yy, zz, xy, xz, yz).  Any pointer may be NULL. */
int rt_moments(rt_state *s, double *E, double *F, double *P, int on_device);

/* Conserved totals (Sec. 2.3.1), deterministic double-precision sums, host
 * output out[16]:
 *   0 sum V e, 1 sum V (c/cbar) E_r, 2 sum V ext_e,
 *   3..5 sum V m, 6..8 sum V F_r / (c cbar), 9..11 sum V ext_m,
 *   12 = 0 + 1 + 2 (conserved), 13..15 = momentum totals (conserved). */
int rt_totals(rt_state *s, double out[16]);

/* The totals of rt_totals, for callers that cannot allocate device memory
 * (no counterpart in the paper: the paper has no GPU).  rt_totals sums into a
 * buffer that rt_create allocated; this call keeps its partial sums and
 * result in one static device array of the library (197 KB on every device
 * that loads it, kept until exit), so the call itself allocates nothing --
 * for code that runs where cudaMalloc is not allowed, or whose device
 * memory belongs to another allocator.  At most 8,388,608 cells; larger
 * states return RT_ERR_ARG.  The same kernels as rt_totals compute the sums:
 * up to 131,072 cells in rt_totals' blocks (bit-identical results), beyond
 * that in larger blocks (the same totals to rounding, not bit for bit).  The
 * first call in a context looks up the array's address
 * (cudaGetSymbolAddress, with that device current): make it before any
 * stream capture; a call in a new context (after cudaDeviceReset, say)
 * looks it up again.  All calls on a device share the array, so calls
 * whose GPU work overlaps race; each call rewrites everything it reads.
 * Synchronises the state's stream; does not report the latched per-cell
 * status (rt_sync does).  out: host, 16 doubles, layout of rt_totals. */
int rt_totals_noalloc(rt_state *s, double out[16]);

/* Waits for the state's stream and rt_step_io's result copies, and returns
 * the latched per-cell status. */
int rt_sync(rt_state *s);

/* Discrete adjoint of one full step (the reverse of rt_step): given the
 * step's forward inputs I^n[N][A], e^n[N], m^n[N][3] (as saved before the
 * step, e.g. by a checkpoint) and the cotangents of its outputs
 * lam_I1 = dL/dI^{n+1}, lam_e1 = dL/de^{n+1}, lam_m1 = dL/dm^{n+1}, writes
 * lam_I = dL/dI^n, lam_e, lam_m and ADDS dL/dkappa_P and dL/dkappa_J (per
 * cell, per unit mass) into grad_kappa_P, grad_kappa_J.  Transport
 * (Sec. 2.2) is linear, its adjoint the transposed upwind gather; the source
 * (Sec. 2.3) is reversed statement by statement, the quartic's root through
 * the implicit-function theorem.  Boundary / emitter tallies carry no
 * cotangent.  Intensities in the state precision, everything else double,
 * caller order; on_device = 1: all arrays are device pointers.  dt <= 0:
 * dt_cfl.  lam_e may alias lam_e1 and lam_m alias lam_m1 (each cell's
 * cotangents are read before its outputs are written); no other arrays may
 * overlap.  The first call allocates the adjoint's work buffers (8 intensity
 * arrays + 35 doubles per cell), kept until rt_destroy. */
int rt_adjoint_step(rt_state *s, double dt, const void *I_n, const double *e_n, const double *m_n,
                    const void *lam_I1, const double *lam_e1, const double *lam_m1, void *lam_I,
                    double *lam_e, double *lam_m, double *grad_kappa_P, double *grad_kappa_J,
                    int on_device);

/* Gas dynamics (states created with params.hydro = 1; Sec. 2, Eq. time
 * evolution with the Euler fluxes): one hydro step of the gas density rho,
 * momentum m and total energy e over dt -- every face's flux the HLLC flux
 * (Toro, Sec. 10.4) of the states on its two sides in the face normal
 * frame, applied to both cells with opposite signs (mass, momentum and
 * energy conserved to rounding); order 1 with the cell-centred states,
 * order 2 the paper's van Leer step (a half step with the cell-centred
 * states, then the full step with the half-step primitives reconstructed
 * linearly at the face centroids from least-squares, Barth-Jespersen-limited
 * gradients).  The faces are static.  The radiation then sees the new
 * density (the opacities per unit mass of rt_set_gas are kept).  Double
 * precision in every state precision.  Errors: RT_ERR_STATE (no hydro or
 * no rt_set_gas), RT_ERR_ARG (dt not positive and finite, order not 1 or
 * 2), RT_ERR_NONFINITE (a density or pressure became non-positive; the gas
 * is then not usable). */
int rt_hydro_step(rt_state *s, double dt, int32_t order);

/* The gas Courant step: cfl * min over cells of V^(1/3) / (|v| + sound
 * speed).  Same requirements as rt_hydro_step. */
int rt_hydro_dt(rt_state *s, double cfl, double *dt);

/* One radiation-hydrodynamics step: rt_hydro_step over dt, then n_sub >= 1
 * radiation steps (transport and implicit source, exchanging energy and
 * momentum with the updated gas) of dt / n_sub each -- the radiation
 * subcycled under the hydro step, as the reduced speed of light allows
 * (Sec. 2, Sec. 3.6).  The radiation steps are checked against the upwind
 * positivity limit like rt_run (RT_ERR_CFL); *dt_rad (may be NULL)
 * receives dt / n_sub.  Per-cell failures are returned as by rt_run. */
int rt_radhydro_step(rt_state *s, double dt, int32_t n_sub, int32_t order, double *dt_rad);

/* The gas density rho[N] (caller order) of a state, host or device
 * pointer. */
int rt_get_density(rt_state *s, double *rho, int on_device);

/* Serialises the full evolving state (intensities, gas e and m, tallies) to
 * a host buffer.  buf == NULL: *bytes receives the size needed. */
int rt_get_state(rt_state *s, void *buf, size_t *bytes);
int rt_set_state(rt_state *s, const void *buf, size_t bytes);

/* Device memory used by the state, in bytes. */
int rt_device_bytes(const rt_state *s, size_t *bytes);

/* Number of kernel launches made by this state since creation. */
int64_t rt_launch_count(const rt_state *s);

const char *rt_last_error(const rt_state *s);
void rt_destroy(rt_state *s);

#ifdef __cplusplus
}
#endif
#endif /* RT_GB300_H */
