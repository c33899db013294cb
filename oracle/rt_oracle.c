/*
 * FP64 CPU oracle of the reduced-speed-of-light radiation step on a Voronoi
 * mesh (Chang, Davis & Jiang, "Time dependent radiation hydrodynamics on a
 * moving mesh").
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code with the CUDA
 * path: it is a plain loop nest written from the paper's equations, in the
 * order the paper gives them, in double precision.
 *
 * Units and readings (the paper leaves these open; see the notes per
 * function): intensities are stored as energy density per steradian, so an
 * isotropic equilibrium field has I = a T^4 / (4 pi); E_r = 4 pi sum_a w_a I_a,
 * F_r = 4 pi c sum_a w_a n_a I_a; the weights sum to one.  The frame velocity
 * of a cell is v = (rho v) / rho at the start of the source step.  The
 * frequency ratio of Sec. 2.3, Gamma_a = gamma (1 - v . n_a / c), is taken
 * to first order in v/c (gamma = 1) unless the problem asks for the
 * transformation to all orders (boost_all_orders, gamma = (1 - v^2/c^2)^-1/2).
 *
 * Every function below is pinned by the CPU tests against something other
 * than itself: closed forms, conservation invariants, brute force on tiny
 * inputs, an mpmath root, the paper's worked example (Sec. 3.1), the
 * diffusion and linear-mode limits (Sec. 3.3, 3.6), geometry identities and
 * exactness on linear fields (the gradient), and orders of accuracy (the
 * van Leer step).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NONCONV (-6)
#define ORC_ERR_NONFINITE (-7)

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  int64_t n_cells, n_faces;
  int32_t n_angles;
  int32_t newton_max_iter;
  /* mesh (Sec. 2, finite-volume charges; Sec. 2.2 transport) */
  const double *cell_volume;  /* [N] */
  const int32_t *face_cells;  /* [Nf][2] */
  const double *face_area;    /* [Nf] */
  const double *face_normal;  /* [Nf][3], unit, i -> j */
  const double *face_w;       /* [Nf][3] face velocity, may be NULL */
  const int64_t *cell_face_ptr; /* [N+1] */
  const int32_t *cell_face_idx; /* [nnz]: f (first cell) or -(f+1) (second) */
  const double *dir;          /* [A][3] */
  const double *wt;           /* [A], sum 1 */
  /* constants */
  double cbar, c, a_rad, gamma_gas, r_gas;
  /* gas, per cell (Sec. 2.3) */
  const double *rho, *kappa_P, *kappa_J, *kappa_s;
  /* boundary / emitter cells (Sec. 2.4, 2.5) */
  const uint8_t *kind;        /* 0 interior, 1 boundary, 2 emitter */
  const double *tau;          /* [N] */
  const double *emit_rate;    /* [N] rho kappa of the emitter */
  const double *I_src;        /* [N] */
  const int32_t *bc_row;      /* [N] */
  const double *I0;           /* [rows][A] */
  /* linear reconstruction: face f = (i, j) -> (x_f - x_i, x_f - x_j'), the
   * face centroid relative to each cell's centroid, j' the image of j that
   * meets i across f; [Nf][2][3], may be NULL when no reconstruction is used */
  const double *face_offset;
  /* 1: Gamma_a = gamma (1 - v . n_a / c) with the Lorentz factor gamma of the
   * frame velocity (the comoving transformation to all orders, Sec. 2.3);
   * 0: gamma = 1 (first order in v/c) */
  int32_t boost_all_orders;
  /* 1: the cells' volumes change with the face velocities by the discrete
   * geometric conservation law (see orc_gcl_volumes) and the transport takes
   * the conservative moving-cell form; cell_volume holds V^n */
  int32_t gcl;
  /* temperature-dependent opacities (Sec. 2.3 solves the temperature
   * equation by Newton-Raphson for them): kappa_P(T) = kappa_P (T/T_ref)^beta_P
   * at T^{n+1} inside the solve, kappa_J(T) = kappa_J (T/T_ref)^beta_J at T^n
   * (the start of the source step); beta_P >= -3.  0, 0: constant opacities */
  double beta_P, beta_J, T_ref;
  /* frequency groups (Sec. 2.3, "multiple independent frequency groups"):
   * n_groups > 1 takes the angle set as n_groups copies of a base set of
   * n_angles / n_groups directions, group j holding angles [j A_g, (j+1) A_g)
   * with weights group_w[j] w_a (the weights of one group sum to group_w[j]);
   * kappa_P, kappa_J, kappa_s then hold n_groups values per cell.  The groups
   * couple only through T^{n+1} (Eq. com rad thermal disc); 1: grey */
  int32_t n_groups;
  const double *group_w;
} orc_problem;

/* ------------------------------------------------------------------------
 * Transport, Sec. 2.2 with the finite-volume update of Eq. (time evolution):
 * the flux through a face moving with velocity w is (cbar n_a - w) . n_f A I
 * and takes I from the upwind side.  Outward flux leaves the cell:
 *   I*_ca = I_ca - dt / V_c * sum_{f in cell c} u_fa I_up,
 *   u_fa = cbar A_f n_a . n_f - A_f w_f . n_f   (n_f outward from c),
 *   I_up = I_ca if u_fa > 0, I_(nbr,a) if u_fa < 0, no flux if u_fa = 0.
 * Faces are visited in the order of the cell's face list.
 * --------------------------------------------------------------------- */
static inline void face_side(const orc_problem *p, int64_t c, int32_t e, int64_t *f,
                             double *sgn, int64_t *nbr) {
  if (e >= 0) {
    *f = e;
    *sgn = 1.0;
    *nbr = p->face_cells[2 * (int64_t)e + 1];
  } else {
    *f = -(int64_t)e - 1;
    *sgn = -1.0;
    *nbr = p->face_cells[2 * (*f)];
  }
  (void)c;
}

/* Rate of change of the volume of cell c, sum_f A_f w_f . n_f (n_f outward),
 * over the cell's faces in list order: with it the discrete geometric
 * conservation law V^{n+1} = V^n + dt sum_f A_f w_f . n_f keeps a uniform
 * field uniform on a moving mesh (Sec. 2.2: the flux through a moving face
 * is (cbar n_a - w) . n_f A I, so a uniform I loses dt I sum_f A (cbar n_a - w)
 * . n_f = -dt I sum_f A w . n_f, which the volume change absorbs). */
static double gcl_rate(const orc_problem *p, int64_t c) {
  double r = 0.0;
  if (!p->face_w) return 0.0;
  for (int64_t k = p->cell_face_ptr[c]; k < p->cell_face_ptr[c + 1]; ++k) {
    int64_t f, nbr;
    double sgn;
    face_side(p, c, p->cell_face_idx[k], &f, &sgn, &nbr);
    const double *nf = p->face_normal + 3 * f, *w = p->face_w + 3 * f;
    r += p->face_area[f] * (sgn * (w[0] * nf[0] + w[1] * nf[1] + w[2] * nf[2]));
  }
  return r;
}

/* V^{n+1} of every cell (the discrete geometric conservation law). */
void orc_gcl_volumes(const orc_problem *p, double dt, double *V_next) {
  for (int64_t c = 0; c < p->n_cells; ++c) V_next[c] = p->cell_volume[c] + dt * gcl_rate(p, c);
}

/* Cells [c0, c1) only; arrays are indexed by global cell number.  With the
 * geometric conservation law (p->gcl) the update is the conservative form
 * for a cell whose volume goes from V^n to V^{n+1} during the step:
 *   V^{n+1} I*_ca = V^n I_ca - dt sum_f u_fa I_up. */
void orc_transport_range(const orc_problem *p, double dt, const double *I, double *Istar,
                         int64_t c0, int64_t c1) {
  const int A = p->n_angles;
#pragma omp parallel for schedule(static)
  for (int64_t c = c0; c < c1; ++c) {
    const double V = p->cell_volume[c];
    const double V1 = p->gcl ? V + dt * gcl_rate(p, c) : V;
    for (int a = 0; a < A; ++a) {
      const double *na = p->dir + 3 * a;
      double acc = 0.0;
      for (int64_t k = p->cell_face_ptr[c]; k < p->cell_face_ptr[c + 1]; ++k) {
        int64_t f, nbr;
        double sgn;
        face_side(p, c, p->cell_face_idx[k], &f, &sgn, &nbr);
        const double *nf = p->face_normal + 3 * f;
        double area = p->face_area[f];
        double ndotn = sgn * (na[0] * nf[0] + na[1] * nf[1] + na[2] * nf[2]);
        double wdotn = 0.0;
        if (p->face_w) {
          const double *w = p->face_w + 3 * f;
          wdotn = sgn * (w[0] * nf[0] + w[1] * nf[1] + w[2] * nf[2]);
        }
        double u = p->cbar * area * ndotn - area * wdotn;
        if (u > 0.0)
          acc += u * I[c * A + a];
        else if (u < 0.0)
          acc += u * I[nbr * A + a];
      }
      if (p->gcl)
        Istar[c * A + a] = (V * I[c * A + a] - dt * acc) / V1;
      else
        Istar[c * A + a] = I[c * A + a] - dt / V * acc;
    }
  }
}

void orc_transport(const orc_problem *p, double dt, const double *I, double *Istar) {
  orc_transport_range(p, dt, I, Istar, 0, p->n_cells);
}

/* Lab-frame moments, Eqs. (moments energy) and (moments flux), with the
 * pressure tensor of Sec. 2.1: E = 4 pi sum w I, F = 4 pi c sum w n I,
 * P = 4 pi sum w n n I (xx, yy, zz, xy, xz, yz). */
static void cell_moments(const orc_problem *p, const double *Ic, double *E, double *F) {
  double e = 0, fx = 0, fy = 0, fz = 0;
  for (int a = 0; a < p->n_angles; ++a) {
    double wi = p->wt[a] * Ic[a];
    e += wi;
    fx += wi * p->dir[3 * a];
    fy += wi * p->dir[3 * a + 1];
    fz += wi * p->dir[3 * a + 2];
  }
  *E = 4.0 * M_PI * e;
  F[0] = 4.0 * M_PI * p->c * fx;
  F[1] = 4.0 * M_PI * p->c * fy;
  F[2] = 4.0 * M_PI * p->c * fz;
}

/* Energy and momentum the radiation of one cell loses in the source step,
 * E^n - E^{n+1} and F^n - F^{n+1}.  The moments are linear in I, so these
 * are 4 pi sum_a w_a dI_a and 4 pi c sum_a w_a n_a dI_a with dI_a = I_a -
 * I'_a, the change of each intensity.  The callers evaluate dI_a as the
 * source term itself (the right side of the discretised equation times dt,
 * see source_interior), not as the difference of the two intensities: where
 * a cell is optically thin the change is a small fraction of I_a, and the
 * difference of two rounded intensities would carry a rounding error of
 * I_a's size, not of the change's. */
static void cell_moment_sum(const orc_problem *p, const double *dI, double *dE, double *dF) {
  double e = 0, fx = 0, fy = 0, fz = 0;
  for (int a = 0; a < p->n_angles; ++a) {
    double wi = p->wt[a] * dI[a];
    e += wi;
    fx += wi * p->dir[3 * a];
    fy += wi * p->dir[3 * a + 1];
    fz += wi * p->dir[3 * a + 2];
  }
  *dE = 4.0 * M_PI * e;
  dF[0] = 4.0 * M_PI * p->c * fx;
  dF[1] = 4.0 * M_PI * p->c * fy;
  dF[2] = 4.0 * M_PI * p->c * fz;
}

void orc_moments(const orc_problem *p, const double *I, double *E, double *F, double *P) {
  const int A = p->n_angles;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < p->n_cells; ++c) {
    const double *Ic = I + c * A;
    double f3[3];
    cell_moments(p, Ic, &E[c], f3);
    if (F) {
      F[3 * c] = f3[0];
      F[3 * c + 1] = f3[1];
      F[3 * c + 2] = f3[2];
    }
    if (P) {
      double s[6] = {0, 0, 0, 0, 0, 0};
      for (int a = 0; a < A; ++a) {
        const double *n = p->dir + 3 * a;
        double wi = p->wt[a] * Ic[a];
        s[0] += wi * n[0] * n[0];
        s[1] += wi * n[1] * n[1];
        s[2] += wi * n[2] * n[2];
        s[3] += wi * n[0] * n[1];
        s[4] += wi * n[0] * n[2];
        s[5] += wi * n[1] * n[2];
      }
      for (int k = 0; k < 6; ++k) P[6 * c + k] = 4.0 * M_PI * s[k];
    }
  }
}

/* ------------------------------------------------------------------------
 * Gas temperature after the implicit step: the unique positive root of
 *   alpha T^4 + beta T - g = 0,  alpha >= 0, beta > 0, g >= 0,
 * which Eq. (com rad thermal disc) becomes once Eq. (Jcom) eliminates J.
 * Newton from T0 = min(g / beta, (g / alpha)^(1/4)), where f(T0) >= 0; f is
 * increasing and convex on T > 0, so the iterates decrease monotonically to
 * the root.  Stops when an iterate fails to decrease or moves by at most
 * 1e-15 of itself.
 * --------------------------------------------------------------------- */
int orc_newton(double alpha, double beta, double g, int max_iter, double *T_out,
               int *iters_out) {
  if (!(alpha >= 0.0) || !(beta > 0.0) || !(g >= 0.0)) return ORC_ERR_NONFINITE;
  double T = g / beta;
  if (alpha > 0.0) {
    double t4 = sqrt(sqrt(g / alpha));
    if (t4 < T) T = t4;
  }
  int it = 0, done = 0;
  while (!done && it < max_iter) {
    double T2 = T * T;
    double f = alpha * T2 * T2 + beta * T - g;
    double fp = 4.0 * alpha * T2 * T + beta;
    double Tn = T - f / fp;
    ++it;
    if (!(Tn < T)) {
      done = 1;
    } else {
      done = (T - Tn <= 1e-15 * T);
      T = Tn;
    }
  }
  if (iters_out) *iters_out = it;
  *T_out = T;
  if (!isfinite(T)) return ORC_ERR_NONFINITE;
  if (!done) return ORC_ERR_NONCONV;
  return ORC_OK;
}

/* Positive root of alpha T^k + beta T = g for k >= 1 (the temperature
 * equation with kappa_P proportional to T^(k-4)), by Newton-Raphson: the
 * left side is increasing and convex for T >= 0, so from the upper bound
 * min(g / beta, (g / alpha)^(1/k)) the iterates decrease monotonically onto
 * the root.  Same stopping rule as orc_newton. */
int orc_newton_power(double alpha, double k, double beta, double g, int max_iter, double *T_out,
                     int *iters_out) {
  if (!(alpha >= 0.0) || !(beta > 0.0) || !(g >= 0.0) || !(k >= 1.0)) return ORC_ERR_NONFINITE;
  double T = g / beta;
  if (alpha > 0.0) {
    double tk = pow(g / alpha, 1.0 / k);
    if (tk < T) T = tk;
  }
  int it = 0, done = 0;
  while (!done && it < max_iter) {
    double Tk1 = pow(T, k - 1.0);
    double f = alpha * Tk1 * T + beta * T - g;
    double fp = k * alpha * Tk1 + beta;
    double Tn = T - f / fp;
    ++it;
    if (!(Tn < T)) {
      done = 1;
    } else {
      done = (T - Tn <= 1e-15 * T);
      T = Tn;
    }
  }
  if (iters_out) *iters_out = it;
  *T_out = T;
  if (!isfinite(T)) return ORC_ERR_NONFINITE;
  if (!done) return ORC_ERR_NONCONV;
  return ORC_OK;
}

/* The opacity factor (T / T_ref)^beta (1 for beta = 0). */
static double opacity_factor(double beta, double T, double T_ref) {
  return beta == 0.0 ? 1.0 : pow(T / T_ref, beta);
}

/* The same root in closed form (Sec. 2.3 solves the temperature-independent
 * case analytically), by Ferrari's method: with p = beta/alpha, q = g/alpha,
 * T^4 + p T - q = 0 is rewritten (T^2 + y)^2 = 2y (T - p/(4y))^2 where y > 0
 * solves the resolvent cubic y^3 + q y - p^2/8 = 0, so the positive root
 * solves T^2 + sqrt(2y) T + y - p / (2 sqrt(2y)) = 0.  Used only as an
 * independent cross-check of the Newton root. */
double orc_ferrari(double alpha, double beta, double g) {
  if (alpha <= 0.0) return g / beta;
  if (g <= 0.0) return 0.0;
  double p = beta / alpha, q = g / alpha;
  double r = p * p / 8.0;
  /* y^3 + q y - r = 0 has a single real root (q > 0); Cardano */
  double disc = sqrt(r * r / 4.0 + q * q * q / 27.0);
  double u = cbrt(r / 2.0 + disc);
  /* second Cardano term -q/(3u) written as the conjugate product form */
  double y = u - q / (3.0 * u);
  if (y <= 0.0) {
    /* fall back: Newton on the cubic from the Cardano estimate */
    y = cbrt(r);
  }
  for (int k = 0; k < 3; ++k) {
    double fy = (y * y + q) * y - r;
    double fpy = 3.0 * y * y + q;
    y -= fy / fpy;
  }
  double s2 = sqrt(2.0 * y);
  double d = -2.0 * y + 2.0 * p / s2;
  double sd = sqrt(d > 0 ? d : 0.0);
  /* T = (-s2 + sd) / 2 = (d - s2^2) / (2 (sd + s2)) */
  return (d - 2.0 * y) / (2.0 * (sd + s2));
}

/* ------------------------------------------------------------------------
 * Implicit source step of one cell, Sec. 2.3, the four-step algorithm:
 *  1. E^n, F^n of the post-transport intensities (Eqs. moments);
 *  2. to the comoving frame: Gamma_a = 1 - v . n_a / c,
 *     I~_a = Gamma_a^4 I_a (Eq. I lab to com), w~_a = N w_a / Gamma_a^2,
 *     sum w~ = 1; the angular sums of Eq. (Jcom) with rho kept:
 *        x_a = dt cbar rho (kJ + ks) Gamma_a,
 *        S_I = sum w~_a I~_a / (1 + x_a),  S_G = sum w~_a Gamma_a / (1 + x_a),
 *        J~ = (S_I + dt cbar rho kP (a T^4 / 4pi) S_G) / D,
 *        D  = 1 - dt cbar rho ks S_G;
 *     eliminating J~ from Eq. (com rad thermal disc) leaves
 *        alpha T^4 + beta T = g,
 *        alpha = dt c rho kP a (1 - dt cbar rho kJ S_G / D),
 *        beta  = rho c_v,  c_v = R / (gamma - 1),
 *        g     = rho c_v T^n + dt c rho 4 pi kJ S_I / D
 *     (D and the bracket of alpha evaluated through S_1 = sum w~ / (1 + x),
 *     see the code);
 *  3. I~^{n+1} from Eq. (com radiative source disc), back to the lab frame;
 *  4. E^{n+1}, F^{n+1} and the gas exchange of Eqs. (gas1), (gas2):
 *        e += (c / cbar)(E^n - E^{n+1}),  rho v += (F^n - F^{n+1}) / (c cbar),
 *     summed angle by angle over the changes dI_a = I_a - I'_a, each taken
 *     from Eq. (com radiative source disc) as the implicit source term:
 *        I~_a - I~'_a = (x_a I~_a - dt cbar Gamma_a rho (kP B + ks J~)) / (1 + x_a),
 *     and dI_a = (I~_a - I~'_a) / Gamma_a^4 (cell_moment_sum).
 * The gas temperature is recomputed from the updated energy next step.
 * --------------------------------------------------------------------- */
/* The Lorentz factor in Gamma_a = gamma (1 - v . n_a / c) (Sec. 2.3): 1 for
 * the first-order transformation. */
static double frame_gamma(const orc_problem *p, const double *v) {
  if (!p->boost_all_orders) return 1.0;
  const double b2 = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / (p->c * p->c);
  return 1.0 / sqrt(1.0 - b2);
}

static int source_interior(const orc_problem *p, int64_t c, double dt, const double *Is,
                           double *In, double *e, double *m, int *iters) {
  const int A = p->n_angles;
  const double rho = p->rho[c], kS = p->kappa_s[c];
  double kin = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho;
  double rcv = rho * p->r_gas / (p->gamma_gas - 1.0);
  double Tn = (*e - kin) / rcv;
  /* kappa_J at the start of the step; kappa_P at T^{n+1} below */
  const double kJ = p->kappa_J[c] * opacity_factor(p->beta_J, Tn, p->T_ref);
  double kP = p->kappa_P[c];
  double v[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
  const double gam = frame_gamma(p, v);
  double G[A], wc[A], Ic[A];
  double norm = 0.0;
  for (int a = 0; a < A; ++a) {
    const double *n = p->dir + 3 * a;
    G[a] = gam * (1.0 - (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / p->c);
    double G2 = G[a] * G[a];
    Ic[a] = G2 * G2 * Is[a];
    wc[a] = p->wt[a] / G2;
    norm += wc[a];
  }
  double SI = 0.0, SG = 0.0, S1 = 0.0;
  for (int a = 0; a < A; ++a) {
    wc[a] /= norm;
    double xa = dt * p->cbar * rho * (kJ + kS) * G[a];
    SI += wc[a] * Ic[a] / (1.0 + xa);
    SG += wc[a] * G[a] / (1.0 + xa);
    S1 += wc[a] / (1.0 + xa);
  }
  /* D = 1 - dt cbar rho ks S_G and 1 - dt cbar rho kJ S_G / D, evaluated
   * through S_1 = sum w~ / (1 + x_a): since the w~ sum to one,
   *   1 - dt cbar rho (kJ + ks) S_G = S_1,  so D = S_1 + dt cbar rho kJ S_G
   * and 1 - dt cbar rho kJ S_G / D = S_1 / D.  The printed forms subtract
   * x / (1 + x) from one and lose log2(x) bits where cells are optically
   * thick (x ~ 1e4 per step in the Sec. 3.1 example with kappa = 100). */
  double D = S1 + dt * p->cbar * rho * kJ * SG;
  double alpha = dt * p->c * rho * kP * p->a_rad * (S1 / D);
  double beta = rcv;
  double g = rcv * Tn + dt * p->c * rho * 4.0 * M_PI * kJ * SI / D;
  double T;
  int st;
  if (p->beta_P == 0.0) {
    st = orc_newton(alpha, beta, g, p->newton_max_iter, &T, iters);
  } else {
    /* kappa_P (T/T_ref)^beta_P T^4 = kappa_P T_ref^-beta_P T^(4 + beta_P) */
    st = orc_newton_power(alpha * pow(p->T_ref, -p->beta_P), 4.0 + p->beta_P, beta, g,
                          p->newton_max_iter, &T, iters);
    kP *= opacity_factor(p->beta_P, T, p->T_ref);
  }
  if (st != ORC_OK) return st;
  double B = p->a_rad * T * T * T * T / (4.0 * M_PI);
  double J = (SI + dt * p->cbar * rho * kP * B * SG) / D;
  double dI[A];
  for (int a = 0; a < A; ++a) {
    double xa = dt * p->cbar * rho * (kJ + kS) * G[a];
    double src = dt * p->cbar * G[a] * rho * (kP * B + kS * J);
    double Inew = (Ic[a] + src) / (1.0 + xa);
    double G2 = G[a] * G[a];
    In[a] = Inew / (G2 * G2);
    dI[a] = ((xa * Ic[a] - src) / (1.0 + xa)) / (G2 * G2);
  }
  double dE, dF[3];
  cell_moment_sum(p, dI, &dE, dF);
  *e += p->c / p->cbar * dE;
  for (int k = 0; k < 3; ++k) m[k] += dF[k] / (p->c * p->cbar);
  return ORC_OK;
}

/* The implicit source step of one interior cell with n_groups > 1
 * frequency groups, Sec. 2.3 generalised to groups j: per group the
 * comoving sums S_I,j and S_G,j over the group's angles (weights normalised
 * within the group), D_j = 1 - dt cbar rho ks_j S_G,j, and Eq. (Jcom) for
 * J~_j; Eq. (com rad thermal disc) weights the groups by W_j:
 *   alpha = sum_j W_j dt c rho kP_j a (1 - dt cbar rho kJ_j S_G,j / D_j),
 *   g     = rho c_v T^n + sum_j W_j dt c rho 4 pi kJ_j S_I,j / D_j,
 * and each group's intensities follow Eq. (com radiative source disc) with
 * its own opacities.  The gas exchange sums all angles with the weights
 * W_j w_a (Eqs. gas1, gas2 with the group weights). */
static int source_interior_groups(const orc_problem *p, int64_t c, double dt, const double *Is,
                                  double *In, double *e, double *m, int *iters) {
  const int A = p->n_angles, NG = p->n_groups, Ag = A / NG;
  const double rho = p->rho[c];
  double kin = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho;
  double rcv = rho * p->r_gas / (p->gamma_gas - 1.0);
  double Tn = (*e - kin) / rcv;
  double v[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
  const double gam = frame_gamma(p, v);
  double G[A], Ic[A], SI[NG], SG[NG], D[NG], kP[NG], kJ[NG], kS[NG];
  double alpha = 0.0, g = rcv * Tn;
  for (int j = 0; j < NG; ++j) {
    kP[j] = p->kappa_P[c * NG + j];
    kJ[j] = p->kappa_J[c * NG + j] * opacity_factor(p->beta_J, Tn, p->T_ref);
    kS[j] = p->kappa_s[c * NG + j];
    double wc[Ag], norm = 0.0;
    for (int b = 0; b < Ag; ++b) {
      const int a = j * Ag + b;
      const double *n = p->dir + 3 * a;
      G[a] = gam * (1.0 - (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / p->c);
      double G2 = G[a] * G[a];
      Ic[a] = G2 * G2 * Is[a];
      wc[b] = p->wt[a] / G2;
      norm += wc[b];
    }
    SI[j] = SG[j] = 0.0;
    double S1 = 0.0;
    for (int b = 0; b < Ag; ++b) {
      const int a = j * Ag + b;
      wc[b] /= norm;
      double xa = dt * p->cbar * rho * (kJ[j] + kS[j]) * G[a];
      SI[j] += wc[b] * Ic[a] / (1.0 + xa);
      SG[j] += wc[b] * G[a] / (1.0 + xa);
      S1 += wc[b] / (1.0 + xa);
    }
    /* D_j and 1 - dt cbar rho kJ_j S_G,j / D_j through S_1 (see source_interior) */
    D[j] = S1 + dt * p->cbar * rho * kJ[j] * SG[j];
    const double W = p->group_w[j];
    alpha += W * dt * p->c * rho * kP[j] * p->a_rad * (S1 / D[j]);
    g += W * dt * p->c * rho * 4.0 * M_PI * kJ[j] * SI[j] / D[j];
  }
  double T;
  int st;
  if (p->beta_P == 0.0) {
    st = orc_newton(alpha, rcv, g, p->newton_max_iter, &T, iters);
  } else {
    st = orc_newton_power(alpha * pow(p->T_ref, -p->beta_P), 4.0 + p->beta_P, rcv, g,
                          p->newton_max_iter, &T, iters);
    for (int j = 0; j < NG; ++j) kP[j] *= opacity_factor(p->beta_P, T, p->T_ref);
  }
  if (st != ORC_OK) return st;
  double B = p->a_rad * T * T * T * T / (4.0 * M_PI);
  double dI[A];
  for (int j = 0; j < NG; ++j) {
    double J = (SI[j] + dt * p->cbar * rho * kP[j] * B * SG[j]) / D[j];
    for (int b = 0; b < Ag; ++b) {
      const int a = j * Ag + b;
      double xa = dt * p->cbar * rho * (kJ[j] + kS[j]) * G[a];
      double src = dt * p->cbar * G[a] * rho * (kP[j] * B + kS[j] * J);
      double Inew = (Ic[a] + src) / (1.0 + xa);
      double G2 = G[a] * G[a];
      In[a] = Inew / (G2 * G2);
      dI[a] = ((xa * Ic[a] - src) / (1.0 + xa)) / (G2 * G2);
    }
  }
  double dE, dF[3];
  cell_moment_sum(p, dI, &dE, dF);
  *e += p->c / p->cbar * dE;
  for (int k = 0; k < 3; ++k) m[k] += dF[k] / (p->c * p->cbar);
  return ORC_OK;
}

/* Boundary cells, Sec. 2.4: I relaxes to I0 with factor min(dt / tau, 1)
 * (tau <= dt pins I = I0).  The gas of a boundary cell is held fixed; the
 * energy and momentum the radiation loses go to an external tally. */
static void source_boundary(const orc_problem *p, int64_t c, double dt, const double *Is,
                            double *In, double *ext) {
  const int A = p->n_angles;
  double f = (p->tau[c] <= dt) ? 1.0 : dt / p->tau[c];
  const double *I0 = p->I0 + (int64_t)p->bc_row[c] * A;
  double dE, dF[3], dI[A];
  for (int a = 0; a < A; ++a) {
    dI[a] = (Is[a] - I0[a]) * f;
    In[a] = Is[a] - dI[a];
  }
  cell_moment_sum(p, dI, &dE, dF);
  ext[0] += p->c / p->cbar * dE;
  for (int k = 0; k < 3; ++k) ext[1 + k] += dF[k] / (p->c * p->cbar);
}

/* Emitter cells, Sec. 2.5: in the comoving frame I~ relaxes implicitly to
 * I_src at rate Gamma_a cbar (rho kappa)_src:
 *   I~^{n+1} = (I~ + y_a I_src) / (1 + y_a),  y_a = dt cbar Gamma_a emit_rate.
 * The emitter's gas is a fixed reservoir; the exchange goes to the tally. */
static void source_emitter(const orc_problem *p, int64_t c, double dt, const double *Is,
                           double *In, const double *m, double *ext) {
  const int A = p->n_angles;
  const double rho = p->rho[c];
  double v[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
  const double gam = frame_gamma(p, v);
  double dE, dF[3], dI[A];
  for (int a = 0; a < A; ++a) {
    const double *n = p->dir + 3 * a;
    double G = gam * (1.0 - (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / p->c);
    double G4 = G * G * G * G;
    double y = dt * p->cbar * G * p->emit_rate[c];
    In[a] = ((G4 * Is[a] + y * p->I_src[c]) / (1.0 + y)) / G4;
    /* the change as the source term: I~ - I~' = y (I~ - I_src) / (1 + y) */
    dI[a] = (y * (G4 * Is[a] - p->I_src[c]) / (1.0 + y)) / G4;
  }
  cell_moment_sum(p, dI, &dE, dF);
  ext[0] += p->c / p->cbar * dE;
  for (int k = 0; k < 3; ++k) ext[1 + k] += dF[k] / (p->c * p->cbar);
}

/* Source step over all cells.  e[N], m[N][3], ext[N][4] are updated in
 * place; Inew may not alias Istar.  Returns the first error met (in cell
 * order) and stores the largest Newton iteration count. */
int orc_source_range(const orc_problem *p, double dt, const double *Istar, double *Inew,
                     double *e, double *m, double *ext, int *max_iters, int64_t c0, int64_t c1) {
  const int A = p->n_angles;
  int status = ORC_OK;
  int64_t first_bad = -1;
  int itmax = 0;
#pragma omp parallel for schedule(static) reduction(max : itmax)
  for (int64_t c = c0; c < c1; ++c) {
    const double *Is = Istar + c * A;
    double *In = Inew + c * A;
    int k = p->kind ? p->kind[c] : 0;
    int it = 0, st = ORC_OK;
    if (k == 1)
      source_boundary(p, c, dt, Is, In, ext + 4 * c);
    else if (k == 2)
      source_emitter(p, c, dt, Is, In, m + 3 * c, ext + 4 * c);
    else
      st = p->n_groups > 1 ? source_interior_groups(p, c, dt, Is, In, e + c, m + 3 * c, &it)
                           : source_interior(p, c, dt, Is, In, e + c, m + 3 * c, &it);
    if (it > itmax) itmax = it;
    for (int a = 0; a < A && st == ORC_OK; ++a)
      if (!isfinite(In[a])) st = ORC_ERR_NONFINITE;
    if (st != ORC_OK) {
#pragma omp critical
      {
        if (first_bad < 0 || c < first_bad) {
          first_bad = c;
          status = st;
        }
      }
    }
  }
  if (max_iters) *max_iters = itmax;
  return status;
}

int orc_source(const orc_problem *p, double dt, const double *Istar, double *Inew, double *e,
               double *m, double *ext, int *max_iters) {
  return orc_source_range(p, dt, Istar, Inew, e, m, ext, max_iters, 0, p->n_cells);
}

/* Transport and source of cells [c0, c1) only, reading I and writing the
 * new intensities of those cells into Iout (global indexing); a bounded
 * sample of one step used to time the oracle. */
int orc_step_range(const orc_problem *p, double dt, const double *I, double *work, double *Iout,
                   double *e, double *m, double *ext, int64_t c0, int64_t c1) {
  orc_transport_range(p, dt, I, work, c0, c1);
  return orc_source_range(p, dt, work, Iout, e, m, ext, NULL, c0, c1);
}

/* One full step: transport over dt, then the implicit source over dt
 * (operator split, forward-Euler transport).  I is replaced by I^{n+1};
 * work[N*A] is scratch. */
int orc_step(const orc_problem *p, double dt, double *I, double *work, double *e, double *m,
             double *ext, int *max_iters) {
  orc_transport(p, dt, I, work);
  return orc_source(p, dt, work, I, e, m, ext, max_iters);
}

/* Courant time step: dt = cfl * min_c V_c^(1/3) / (cbar + max_f |w_f|). */
double orc_cfl_dt(const orc_problem *p, double cfl) {
  double best = INFINITY;
  for (int64_t c = 0; c < p->n_cells; ++c) {
    double wmax = 0.0;
    if (p->face_w)
      for (int64_t k = p->cell_face_ptr[c]; k < p->cell_face_ptr[c + 1]; ++k) {
        int32_t e = p->cell_face_idx[k];
        int64_t f = e >= 0 ? e : -(int64_t)e - 1;
        const double *w = p->face_w + 3 * f;
        double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if (wn > wmax) wmax = wn;
      }
    double d = cbrt(p->cell_volume[c]) / (p->cbar + wmax);
    if (d < best) best = d;
  }
  return cfl * best;
}

/* Positivity of the upwind update: I*_ca keeps a non-negative weight on
 * I_ca iff dt * K_ca <= 1 with K_ca = (1 / V_c) sum_f max(u_fa, 0).
 * Returns max over cells and angles of K_ca. */
double orc_positivity(const orc_problem *p) {
  const int A = p->n_angles;
  double kmax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : kmax)
  for (int64_t c = 0; c < p->n_cells; ++c) {
    for (int a = 0; a < A; ++a) {
      const double *na = p->dir + 3 * a;
      double s = 0.0;
      for (int64_t k = p->cell_face_ptr[c]; k < p->cell_face_ptr[c + 1]; ++k) {
        int64_t f, nbr;
        double sgn;
        face_side(p, c, p->cell_face_idx[k], &f, &sgn, &nbr);
        const double *nf = p->face_normal + 3 * f;
        double area = p->face_area[f];
        double ndotn = sgn * (na[0] * nf[0] + na[1] * nf[1] + na[2] * nf[2]);
        double wdotn = 0.0;
        if (p->face_w) {
          const double *w = p->face_w + 3 * f;
          wdotn = sgn * (w[0] * nf[0] + w[1] * nf[1] + w[2] * nf[2]);
        }
        double u = p->cbar * area * ndotn - area * wdotn;
        if (u > 0.0) s += u;
      }
      s /= p->cell_volume[c];
      if (s > kmax) kmax = s;
    }
  }
  return kmax;
}

/* Conserved totals (Sec. 2.3.1): with E_g the gas energy and the radiation
 * weighted by c / cbar, E_g + (c/cbar) E_r and rho v + F_r / (c cbar) are
 * conserved; the tallies of boundary / emitter cells close the budget.
 * out[0..2]  sum V e, sum V (c/cbar) E_r, sum V ext_e
 * out[3..5]  sum V rho v
 * out[6..8]  sum V F_r / (c cbar)
 * out[9..11] sum V ext_m
 * out[12]    out[0] + out[1] + out[2]
 * out[13..15] total momentum.  Plain sums in cell order. */
void orc_totals(const orc_problem *p, const double *I, const double *e, const double *m,
                const double *ext, double *out) {
  const int A = p->n_angles;
  for (int k = 0; k < 16; ++k) out[k] = 0.0;
  for (int64_t c = 0; c < p->n_cells; ++c) {
    double V = p->cell_volume[c];
    double E, F[3];
    cell_moments(p, I + c * A, &E, F);
    out[0] += V * e[c];
    out[1] += V * (p->c / p->cbar) * E;
    out[2] += ext ? V * ext[4 * c] : 0.0;
    for (int k = 0; k < 3; ++k) {
      out[3 + k] += V * m[3 * c + k];
      out[6 + k] += V * F[k] / (p->c * p->cbar);
      out[9 + k] += ext ? V * ext[4 * c + 1 + k] : 0.0;
    }
  }
  out[12] = out[0] + out[1] + out[2];
  for (int k = 0; k < 3; ++k) out[13 + k] = out[3 + k] + out[6 + k] + out[9 + k];
}

/* ========================================================================
 * Discrete adjoint of one step (the gradient of a scalar loss through
 * transport then source), written out by hand in reverse order of the
 * forward statements above.  The absorption opacity is the parameter:
 * kappa_P and kappa_J each receive a gradient; kappa_s, rho and the mesh are
 * fixed.  Inputs: the step's forward inputs I, e, m and the cotangents
 * lI1 = dL/dI^{n+1}, le1 = dL/de^{n+1}, lm1 = dL/dm^{n+1}.  Outputs:
 * lI = dL/dI^n, le = dL/de^n, lm = dL/dm^n; gP, gJ accumulate (+=)
 * dL/dkappa_P, dL/dkappa_J.  The boundary / emitter tallies are outputs only
 * (no loss depends on them), so they carry no cotangent.
 * --------------------------------------------------------------------- */

/* Transpose of the transport map I* = M I (Sec. 2.2): M is linear in I with
 * M_cc,a = 1 - dt/V_c sum_f max(u_fa, 0) and M_c,nbr,a = -dt/V_c u_fa for
 * the faces where u_fa < 0.  A face outflow of cell j (u_jfa > 0) is the
 * inflow of its neighbour through the same face, so
 *   (M^T l)_ja = l_ja - sum_{f in j, u_jfa > 0} u_jfa (dt/V_j l_ja - dt/V_nbr l_nbr,a). */
void orc_transport_adjoint(const orc_problem *p, double dt, const double *l, double *out) {
  const int A = p->n_angles;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < p->n_cells; ++c) {
    for (int a = 0; a < A; ++a) {
      const double *na = p->dir + 3 * a;
      double acc = 0.0;
      for (int64_t k = p->cell_face_ptr[c]; k < p->cell_face_ptr[c + 1]; ++k) {
        int64_t f, nbr;
        double sgn;
        face_side(p, c, p->cell_face_idx[k], &f, &sgn, &nbr);
        const double *nf = p->face_normal + 3 * f;
        double area = p->face_area[f];
        double ndotn = sgn * (na[0] * nf[0] + na[1] * nf[1] + na[2] * nf[2]);
        double wdotn = 0.0;
        if (p->face_w) {
          const double *w = p->face_w + 3 * f;
          wdotn = sgn * (w[0] * nf[0] + w[1] * nf[1] + w[2] * nf[2]);
        }
        double u = p->cbar * area * ndotn - area * wdotn;
        if (u > 0.0)
          acc += u * (dt / p->cell_volume[c] * l[c * A + a] - dt / p->cell_volume[nbr] * l[nbr * A + a]);
      }
      out[c * A + a] = l[c * A + a] - acc;
    }
  }
}

/* Reverse of source_interior for one cell. */
static void source_interior_adjoint(const orc_problem *p, int64_t c, double dt, const double *Is,
                                    const double *e_in, const double *m, const double *lI1,
                                    double le1, const double *lm1, double *lIs, double *le,
                                    double *lm, double *gP, double *gJ) {
  const int A = p->n_angles;
  const double rho = p->rho[c], kP = p->kappa_P[c], kJ = p->kappa_J[c], kS = p->kappa_s[c];
  const double cb = p->cbar, cc = p->c, ar = p->a_rad;
  /* ---- forward recomputation */
  double v[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
  double G[A], wh[A], wt[A], It[A], x[A], Itn[A], In[A];
  double Nw = 0.0;
  for (int a = 0; a < A; ++a) {
    const double *n = p->dir + 3 * a;
    G[a] = 1.0 - (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / cc;
    It[a] = G[a] * G[a] * G[a] * G[a] * Is[a];
    wh[a] = p->wt[a] / (G[a] * G[a]);
    Nw += wh[a];
  }
  double SI = 0.0, SG = 0.0;
  for (int a = 0; a < A; ++a) {
    wt[a] = wh[a] / Nw;
    x[a] = dt * cb * rho * (kJ + kS) * G[a];
    SI += wt[a] * It[a] / (1.0 + x[a]);
    SG += wt[a] * G[a] / (1.0 + x[a]);
  }
  const double D = 1.0 - dt * cb * rho * kS * SG;
  const double kin = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho;
  const double rcv = rho * p->r_gas / (p->gamma_gas - 1.0);
  const double Tn = (*e_in - kin) / rcv;
  const double hJ = 1.0 - dt * cb * rho * kJ * SG / D;
  const double alpha = dt * cc * rho * kP * ar * hJ;
  const double g = rcv * Tn + dt * cc * rho * 4.0 * M_PI * kJ * SI / D;
  double T;
  orc_newton(alpha, rcv, g, p->newton_max_iter, &T, NULL);
  const double B = ar * T * T * T * T / (4.0 * M_PI);
  const double J = (SI + dt * cb * rho * kP * B * SG) / D;
  const double q = dt * cb * rho * (kP * B + kS * J);
  for (int a = 0; a < A; ++a) {
    Itn[a] = (It[a] + q * G[a]) / (1.0 + x[a]);
    In[a] = Itn[a] / (G[a] * G[a] * G[a] * G[a]);
  }
  /* ---- reverse */
  /* e' = e + (c/cbar) dE, m' = m + dF/(c cbar), dE = 4 pi sum w (I* - I'),
     dF = 4 pi c sum w n (I* - I') */
  const double ldE = cc / cb * le1;
  double ldF[3] = {lm1[0] / (cc * cb), lm1[1] / (cc * cb), lm1[2] / (cc * cb)};
  double lG[A], lIt[A], lx[A], lwt[A];
  double lq = 0.0;
  for (int a = 0; a < A; ++a) {
    const double *n = p->dir + 3 * a;
    const double ex = 4.0 * M_PI * p->wt[a] * (ldE + cc * (n[0] * ldF[0] + n[1] * ldF[1] + n[2] * ldF[2]));
    lIs[a] = ex;                     /* I* enters dE, dF directly */
    const double lIn = lI1[a] - ex;  /* I' enters them with a minus sign */
    const double G4 = G[a] * G[a] * G[a] * G[a];
    const double lItn = lIn / G4;
    lG[a] = -4.0 * In[a] / G[a] * lIn;
    lIt[a] = lItn / (1.0 + x[a]);
    lq += G[a] * lItn / (1.0 + x[a]);
    lG[a] += q * lItn / (1.0 + x[a]);
    lx[a] = -Itn[a] * lItn / (1.0 + x[a]);
  }
  double lB = dt * cb * rho * kP * lq;
  double lJ = dt * cb * rho * kS * lq;
  *gP += dt * cb * rho * B * lq;
  /* J = (SI + dt cbar rho kP B SG) / D */
  double lSI = lJ / D;
  double lSG = dt * cb * rho * kP * B * lJ / D;
  double lD = -J * lJ / D;
  lB += dt * cb * rho * kP * SG * lJ / D;
  *gP += dt * cb * rho * B * SG * lJ / D;
  /* B = a T^4 / 4 pi; T from alpha T^4 + rcv T - g = 0 (implicit function) */
  const double lT = ar * T * T * T / M_PI * lB;
  const double Fp = 4.0 * alpha * T * T * T + rcv;
  const double lalpha = -T * T * T * T / Fp * lT;
  const double lg = lT / Fp;
  /* g = rcv Tn + dt c rho 4 pi kJ SI / D */
  const double lTn = rcv * lg;
  lSI += dt * cc * rho * 4.0 * M_PI * kJ / D * lg;
  lD += -dt * cc * rho * 4.0 * M_PI * kJ * SI / (D * D) * lg;
  *gJ += dt * cc * rho * 4.0 * M_PI * SI / D * lg;
  /* alpha = dt c rho kP a (1 - dt cbar rho kJ SG / D) */
  *gP += dt * cc * rho * ar * hJ * lalpha;
  *gJ += dt * cc * rho * kP * ar * (-dt * cb * rho * SG / D) * lalpha;
  lSG += dt * cc * rho * kP * ar * (-dt * cb * rho * kJ / D) * lalpha;
  lD += dt * cc * rho * kP * ar * (dt * cb * rho * kJ * SG / (D * D)) * lalpha;
  /* Tn = (e - kin) / rcv, kin = |m|^2 / (2 rho) */
  *le = le1 + lTn / rcv;
  const double lkin = -lTn / rcv;
  for (int k = 0; k < 3; ++k) lm[k] = lm1[k] + m[k] / rho * lkin;
  /* D = 1 - dt cbar rho kS SG */
  lSG += -dt * cb * rho * kS * lD;
  /* SI = sum wt It / (1 + x), SG = sum wt G / (1 + x) */
  double swl = 0.0;
  for (int a = 0; a < A; ++a) {
    const double r = 1.0 / (1.0 + x[a]);
    lwt[a] = (It[a] * lSI + G[a] * lSG) * r;
    lIt[a] += wt[a] * lSI * r;
    lG[a] += wt[a] * lSG * r;
    lx[a] += -wt[a] * (It[a] * lSI + G[a] * lSG) * r * r;
    swl += wt[a] * lwt[a];
  }
  double lv[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < A; ++a) {
    /* x = dt cbar rho (kJ + kS) G */
    *gJ += dt * cb * rho * G[a] * lx[a];
    lG[a] += dt * cb * rho * (kJ + kS) * lx[a];
    /* wt = wh / sum wh, wh = w / G^2 */
    const double lwh = (lwt[a] - swl) / Nw;
    lG[a] += -2.0 * wh[a] / G[a] * lwh;
    /* It = G^4 I* */
    lIs[a] += G[a] * G[a] * G[a] * G[a] * lIt[a];
    lG[a] += 4.0 * G[a] * G[a] * G[a] * Is[a] * lIt[a];
    /* G = 1 - v . n / c */
    const double *n = p->dir + 3 * a;
    for (int k = 0; k < 3; ++k) lv[k] += -n[k] / cc * lG[a];
  }
  for (int k = 0; k < 3; ++k) lm[k] += lv[k] / rho;
}

/* Reverse of source_emitter: I'_a = (I*_a + Y I_src G_a^-3) / (1 + Y G_a),
 * Y = dt cbar emit_rate, G_a = 1 - v . n_a / c; the gas is a reservoir. */
static void source_emitter_adjoint(const orc_problem *p, int64_t c, double dt, const double *Is,
                                   const double *m, const double *lI1, double le1,
                                   const double *lm1, double *lIs, double *le, double *lm) {
  const int A = p->n_angles;
  const double rho = p->rho[c];
  const double v[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
  const double Y = dt * p->cbar * p->emit_rate[c];
  double lv[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < A; ++a) {
    const double *n = p->dir + 3 * a;
    const double G = 1.0 - (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / p->c;
    const double G4 = G * G * G * G;
    const double y = Y * G;
    const double In = ((G4 * Is[a] + y * p->I_src[c]) / (1.0 + y)) / G4;
    lIs[a] = lI1[a] / (1.0 + y);
    const double dIdG = (-3.0 * Y * p->I_src[c] / G4 - Y * In) / (1.0 + y);
    for (int k = 0; k < 3; ++k) lv[k] += -n[k] / p->c * dIdG * lI1[a];
  }
  *le = le1;
  for (int k = 0; k < 3; ++k) lm[k] = lm1[k] + lv[k] / rho;
}

/* Adjoint of one full step (transport then source).  work[N*A] x 2 scratch. */
int orc_adjoint_step(const orc_problem *p, double dt, const double *I, const double *e,
                     const double *m, const double *lI1, const double *le1, const double *lm1,
                     double *lI, double *le, double *lm, double *gP, double *gJ, double *work) {
  const int A = p->n_angles;
  double *Is = work, *lIs = work + p->n_cells * A;
  /* reverses the first-order transformation on a mesh of fixed volumes only */
  if (p->boost_all_orders || p->gcl || p->beta_P != 0.0 || p->beta_J != 0.0 || p->n_groups > 1)
    return ORC_ERR_ARG;
  orc_transport(p, dt, I, Is);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < p->n_cells; ++c) {
    const int k = p->kind ? p->kind[c] : 0;
    if (k == 1) {
      const double f = (p->tau[c] <= dt) ? 1.0 : dt / p->tau[c];
      for (int a = 0; a < A; ++a) lIs[c * A + a] = (1.0 - f) * lI1[c * A + a];
      le[c] = le1[c];
      for (int d = 0; d < 3; ++d) lm[3 * c + d] = lm1[3 * c + d];
    } else if (k == 2) {
      source_emitter_adjoint(p, c, dt, Is + c * A, m + 3 * c, lI1 + c * A, le1[c], lm1 + 3 * c,
                             lIs + c * A, le + c, lm + 3 * c);
    } else {
      source_interior_adjoint(p, c, dt, Is + c * A, e + c, m + 3 * c, lI1 + c * A, le1[c],
                              lm1 + 3 * c, lIs + c * A, le + c, lm + 3 * c, gP + c, gJ + c);
    }
  }
  orc_transport_adjoint(p, dt, lIs, lI);
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Limited linear reconstruction and the van Leer two-stage step (Sec. 2,
 * the integration steps with the "van Leer method"; Sec. 2.2, transport
 * step 2: the state at the face centre by linear reconstruction with a
 * limiter).  The paper defers the gradient estimate and the limiter to its
 * hydrodynamics code; this oracle takes (readings):
 *   gradient g of I_a in cell c: least squares over the face neighbours,
 *     minimising sum_f w_f (I_j - I_c - g . r_f)^2 with r_f = x_j' - x_c
 *     (centroid of the neighbour's image across f) and w_f = A_f / |r_f|^2,
 *     i.e. g = M^-1 b, M = sum_f w_f r_f r_f^T, b = sum_f w_f r_f (I_j - I_c);
 *     exact for a linear field;
 *   limiter (Barth-Jespersen): g <- alpha g, alpha the largest value in
 *     [0, 1] keeping I_c + g . (x_f - x_c) within [min, max] of I_c and its
 *     face neighbours on every face of c.
 * --------------------------------------------------------------------- */
static inline void face_offsets(const orc_problem *p, int32_t e, const double **d_own,
                                const double **d_nbr) {
  const int64_t f = e >= 0 ? e : -(int64_t)e - 1;
  const double *o = p->face_offset + 6 * f;
  *d_own = e >= 0 ? o : o + 3;
  *d_nbr = e >= 0 ? o + 3 : o;
}

/* grad[(c * 3 + d) * A + a] = d-th component of the (limited, if limit)
 * gradient of I_a in cell c. */
void orc_gradient(const orc_problem *p, const double *I, int limit, double *grad) {
  const int A = p->n_angles;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < p->n_cells; ++c) {
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int64_t k = p->cell_face_ptr[c]; k < p->cell_face_ptr[c + 1]; ++k) {
      const double *d_own, *d_nbr;
      face_offsets(p, p->cell_face_idx[k], &d_own, &d_nbr);
      int64_t f, nbr;
      double sgn;
      face_side(p, c, p->cell_face_idx[k], &f, &sgn, &nbr);
      double r[3] = {d_own[0] - d_nbr[0], d_own[1] - d_nbr[1], d_own[2] - d_nbr[2]};
      double w = p->face_area[f] / (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
      for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) M[x][y] += w * r[x] * r[y];
    }
    /* inverse of the symmetric 3x3 matrix by cofactors */
    double C[3][3];
    C[0][0] = M[1][1] * M[2][2] - M[1][2] * M[2][1];
    C[0][1] = M[0][2] * M[2][1] - M[0][1] * M[2][2];
    C[0][2] = M[0][1] * M[1][2] - M[0][2] * M[1][1];
    C[1][0] = M[1][2] * M[2][0] - M[1][0] * M[2][2];
    C[1][1] = M[0][0] * M[2][2] - M[0][2] * M[2][0];
    C[1][2] = M[0][2] * M[1][0] - M[0][0] * M[1][2];
    C[2][0] = M[1][0] * M[2][1] - M[1][1] * M[2][0];
    C[2][1] = M[0][1] * M[2][0] - M[0][0] * M[2][1];
    C[2][2] = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    const double det = M[0][0] * C[0][0] + M[0][1] * C[1][0] + M[0][2] * C[2][0];
    for (int a = 0; a < A; ++a) {
      const double Ic = I[c * A + a];
      double b[3] = {0, 0, 0}, lo = Ic, hi = Ic;
      for (int64_t k = p->cell_face_ptr[c]; k < p->cell_face_ptr[c + 1]; ++k) {
        const double *d_own, *d_nbr;
        face_offsets(p, p->cell_face_idx[k], &d_own, &d_nbr);
        int64_t f, nbr;
        double sgn;
        face_side(p, c, p->cell_face_idx[k], &f, &sgn, &nbr);
        double r[3] = {d_own[0] - d_nbr[0], d_own[1] - d_nbr[1], d_own[2] - d_nbr[2]};
        double w = p->face_area[f] / (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        const double Ij = I[nbr * A + a];
        for (int x = 0; x < 3; ++x) b[x] += w * r[x] * (Ij - Ic);
        if (Ij < lo) lo = Ij;
        if (Ij > hi) hi = Ij;
      }
      double g[3];
      for (int x = 0; x < 3; ++x) g[x] = (C[x][0] * b[0] + C[x][1] * b[1] + C[x][2] * b[2]) / det;
      if (limit) {
        double alpha = 1.0;
        for (int64_t k = p->cell_face_ptr[c]; k < p->cell_face_ptr[c + 1]; ++k) {
          const double *d_own, *d_nbr;
          face_offsets(p, p->cell_face_idx[k], &d_own, &d_nbr);
          const double dI = g[0] * d_own[0] + g[1] * d_own[1] + g[2] * d_own[2];
          double al = 1.0;
          if (dI > 0.0) al = (hi - Ic) / dI;
          else if (dI < 0.0) al = (lo - Ic) / dI;
          if (al < alpha) alpha = al;
        }
        for (int x = 0; x < 3; ++x) g[x] *= alpha;
      }
      for (int x = 0; x < 3; ++x) grad[(c * 3 + x) * A + a] = g[x];
    }
  }
}

/* The transport update of I over dt with the upwind value of each face
 * reconstructed from (Ih, grad): I_up = Ih_u + g_u . (x_f - x_u), u the
 * upwind cell (the same face value on both sides of the face). */
void orc_transport_recon(const orc_problem *p, double dt, const double *I, const double *Ih,
                         const double *grad, double *Istar) {
  const int A = p->n_angles;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < p->n_cells; ++c) {
    for (int a = 0; a < A; ++a) {
      const double *na = p->dir + 3 * a;
      double acc = 0.0;
      for (int64_t k = p->cell_face_ptr[c]; k < p->cell_face_ptr[c + 1]; ++k) {
        int64_t f, nbr;
        double sgn;
        face_side(p, c, p->cell_face_idx[k], &f, &sgn, &nbr);
        const double *d_own, *d_nbr;
        face_offsets(p, p->cell_face_idx[k], &d_own, &d_nbr);
        const double *nf = p->face_normal + 3 * f;
        double area = p->face_area[f];
        double ndotn = sgn * (na[0] * nf[0] + na[1] * nf[1] + na[2] * nf[2]);
        double wdotn = 0.0;
        if (p->face_w) {
          const double *w = p->face_w + 3 * f;
          wdotn = sgn * (w[0] * nf[0] + w[1] * nf[1] + w[2] * nf[2]);
        }
        double u = p->cbar * area * ndotn - area * wdotn;
        if (u > 0.0) {
          const double *g = grad + c * 3 * A + a;
          acc += u * (Ih[c * A + a] + (g[0] * d_own[0] + g[A] * d_own[1] + g[2 * A] * d_own[2]));
        } else if (u < 0.0) {
          const double *g = grad + nbr * 3 * A + a;
          acc += u * (Ih[nbr * A + a] + (g[0] * d_nbr[0] + g[A] * d_nbr[1] + g[2 * A] * d_nbr[2]));
        }
      }
      Istar[c * A + a] = I[c * A + a] - dt / p->cell_volume[c] * acc;
    }
  }
}

/* One van Leer step (reading of the integration steps with the van Leer
 * half step):
 *   stage 1: I^{n+1/2} = source_{dt/2}(transport_{dt/2}(I^n)) with
 *            piecewise-constant upwinding, on a copy of the gas (discarded);
 *   stage 2: I* = I^n - dt/V sum_f u I_up(I^{n+1/2}, limited gradients of
 *            I^{n+1/2}), then the implicit source over dt from the gas at n.
 * I is replaced by I^{n+1}; work, Ih [N*A] and grad [N*3*A] are scratch. */
int orc_step_vl(const orc_problem *p, double dt, double *I, double *work, double *Ih,
                double *grad, double *e, double *m, double *ext, int *max_iters) {
  const int64_t N = p->n_cells;
  double *e1 = (double *)malloc(sizeof(double) * N);
  double *m1 = (double *)malloc(sizeof(double) * 3 * N);
  double *x1 = (double *)malloc(sizeof(double) * 4 * N);
  if (!e1 || !m1 || !x1) {
    free(e1);
    free(m1);
    free(x1);
    return ORC_ERR_NONFINITE;
  }
  memcpy(e1, e, sizeof(double) * N);
  memcpy(m1, m, sizeof(double) * 3 * N);
  memcpy(x1, ext, sizeof(double) * 4 * N);
  orc_transport(p, 0.5 * dt, I, work);
  int st = orc_source(p, 0.5 * dt, work, Ih, e1, m1, x1, NULL);
  free(e1);
  free(m1);
  free(x1);
  if (st != ORC_OK) return st;
  orc_gradient(p, Ih, 1, grad);
  orc_transport_recon(p, dt, I, Ih, grad, work);
  return orc_source(p, dt, work, I, e, m, ext, max_iters);
}

/* Threads of the OpenMP loops from now on (n > 0); returns the count in
 * effect.  Lets a caller time the oracle on one core and on all of them in
 * one process. */
int orc_set_threads(int n) {
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
}

/* ===================================================================
 * Hydrodynamics on the mesh (Sec. 2, Eq. time evolution with the Euler
 * fluxes; the Riemann-solver steps of Sec. 2): the gas state per cell is
 * rho, m = rho v and the total energy density e = rho v^2 / 2 + P /
 * (gamma - 1) -- the same e and m the radiation source step exchanges with.
 * Each face's flux is the HLLC flux (Toro, Riemann Solvers and Numerical
 * Methods for Fluid Dynamics, 3rd ed., Sec. 10.4, with the wave-speed
 * estimates of Davis, Sec. 10.5.1) of the states on its two sides, rotated
 * into the face normal n_f (from the face's first cell to its second); the
 * faces are static (the linear-wave test fixes its mesh).  Each face's flux
 * is computed once, from (first cell, second cell, n_f), and enters its two
 * cells with opposite signs, so mass, momentum and energy are conserved to
 * rounding.
 * Time integration (Sec. 2, integration steps): the van Leer step -- a
 * half step over dt/2 with the cell-centred states on both sides of each
 * face, then the full step over dt from the initial state with the fluxes of
 * the half-step primitives (rho, v, P) reconstructed linearly at the face
 * centroids with the least-squares, Barth-Jespersen-limited gradients of
 * orc_gradient (the reading of the gradient and limiter used for the
 * radiation, which the paper takes from its hydrodynamics) -- or, with
 * order 1, one step with the cell-centred states.
 * =================================================================== */

/* primitive (rho, vx, vy, vz, P) of a cell */
static void hydro_prim(double gamma, double rho, const double *m, double e, double *W) {
  W[0] = rho;
  W[1] = m[0] / rho;
  W[2] = m[1] / rho;
  W[3] = m[2] / rho;
  W[4] = (gamma - 1.0) * (e - 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho);
}

/* HLLC flux per unit area of (rho, m, e) through a face with unit normal n,
 * left state WL on the side n points away from.  Returns -1 if a state has
 * non-positive density or pressure. */
int orc_hllc_flux(double gamma, const double *WL, const double *WR, const double *n, double *F) {
  const double *W[2] = {WL, WR};
  double u[2], a[2], E[2], Fk[2][5];
  for (int k = 0; k < 2; ++k) {
    const double *w = W[k];
    if (!(w[0] > 0.0) || !(w[4] > 0.0)) return -1;
    u[k] = w[1] * n[0] + w[2] * n[1] + w[3] * n[2];
    a[k] = sqrt(gamma * w[4] / w[0]);
    E[k] = w[4] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
    Fk[k][0] = w[0] * u[k];
    for (int d = 0; d < 3; ++d) Fk[k][1 + d] = w[0] * w[1 + d] * u[k] + w[4] * n[d];
    Fk[k][4] = (E[k] + w[4]) * u[k];
  }
  /* Davis's estimates of the slowest and fastest signal speeds */
  const double SL = fmin(u[0] - a[0], u[1] - a[1]);
  const double SR = fmax(u[0] + a[0], u[1] + a[1]);
  /* the contact's speed (Toro Eq. 10.37) */
  const double Ss = (WR[4] - WL[4] + WL[0] * u[0] * (SL - u[0]) - WR[0] * u[1] * (SR - u[1])) /
                    (WL[0] * (SL - u[0]) - WR[0] * (SR - u[1]));
  if (SL >= 0.0) {
    for (int q = 0; q < 5; ++q) F[q] = Fk[0][q];
  } else if (SR <= 0.0) {
    for (int q = 0; q < 5; ++q) F[q] = Fk[1][q];
  } else {
    /* the star state of side K (Toro Eq. 10.39, the tangential velocity
     * carried unchanged) and F*_K = F_K + S_K (U*_K - U_K) */
    const int k = (Ss >= 0.0) ? 0 : 1;
    const double S = k == 0 ? SL : SR;
    const double *w = W[k];
    const double f = w[0] * (S - u[k]) / (S - Ss);
    double Us[5], U[5];
    Us[0] = f;
    for (int d = 0; d < 3; ++d) Us[1 + d] = f * (w[1 + d] + (Ss - u[k]) * n[d]);
    Us[4] = f * (E[k] / w[0] + (Ss - u[k]) * (Ss + w[4] / (w[0] * (S - u[k]))));
    U[0] = w[0];
    for (int d = 0; d < 3; ++d) U[1 + d] = w[0] * w[1 + d];
    U[4] = E[k];
    for (int q = 0; q < 5; ++q) F[q] = Fk[k][q] + S * (Us[q] - U[q]);
  }
  return 0;
}

/* cfl * min over cells of V^(1/3) / (|v| + sound speed) */
double orc_hydro_dt(const orc_problem *p, const double *rho, const double *m, const double *e,
                    double cfl) {
  double best = INFINITY;
  for (int64_t c = 0; c < p->n_cells; ++c) {
    double W[5];
    hydro_prim(p->gamma_gas, rho[c], m + 3 * c, e[c], W);
    const double v = sqrt(W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
    const double a = sqrt(p->gamma_gas * W[4] / W[0]);
    const double t = cbrt(p->cell_volume[c]) / (v + a);
    if (t < best) best = t;
  }
  return cfl * best;
}

/* Fluxes of every face (area times HLLC flux, Fa[Nf][5]) from the
 * primitives W[N][5], cell-centred (grad NULL) or reconstructed at the face
 * centroid with grad[N][3][5]: W_i + g_i . (x_f - x_i), W_j + g_j . (x_f - x_j').
 * Returns -1 if a face state is not physical. */
static int hydro_face_fluxes(const orc_problem *p, const double *W, const double *grad,
                             double *Fa) {
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t f = 0; f < p->n_faces; ++f) {
    const int64_t i = p->face_cells[2 * f], j = p->face_cells[2 * f + 1];
    double WL[5], WR[5];
    for (int q = 0; q < 5; ++q) {
      WL[q] = W[i * 5 + q];
      WR[q] = W[j * 5 + q];
    }
    if (grad) {
      const double *oi = p->face_offset + 6 * f, *oj = oi + 3;
      for (int q = 0; q < 5; ++q) {
        WL[q] += grad[(i * 3 + 0) * 5 + q] * oi[0] + grad[(i * 3 + 1) * 5 + q] * oi[1] +
                 grad[(i * 3 + 2) * 5 + q] * oi[2];
        WR[q] += grad[(j * 3 + 0) * 5 + q] * oj[0] + grad[(j * 3 + 1) * 5 + q] * oj[1] +
                 grad[(j * 3 + 2) * 5 + q] * oj[2];
      }
    }
    double F[5];
    if (orc_hllc_flux(p->gamma_gas, WL, WR, p->face_normal + 3 * f, F) != 0) bad = 1;
    for (int q = 0; q < 5; ++q) Fa[f * 5 + q] = p->face_area[f] * F[q];
  }
  return bad ? -1 : 0;
}

/* U_out = U_in - h / V sum over the cell's faces (in list order) of the
 * outward face fluxes (+Fa for the face's first cell, -Fa for its second). */
static void hydro_apply(const orc_problem *p, double h, const double *Fa, const double *rho_in,
                        const double *m_in, const double *e_in, double *rho, double *m,
                        double *e) {
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < p->n_cells; ++c) {
    double s[5] = {0, 0, 0, 0, 0};
    for (int64_t k = p->cell_face_ptr[c]; k < p->cell_face_ptr[c + 1]; ++k) {
      const int32_t ent = p->cell_face_idx[k];
      const int64_t f = ent >= 0 ? ent : -(int64_t)ent - 1;
      const double sg = ent >= 0 ? 1.0 : -1.0;
      for (int q = 0; q < 5; ++q) s[q] += sg * Fa[f * 5 + q];
    }
    const double hv = h / p->cell_volume[c];
    rho[c] = rho_in[c] - hv * s[0];
    for (int d = 0; d < 3; ++d) m[3 * c + d] = m_in[3 * c + d] - hv * s[1 + d];
    e[c] = e_in[c] - hv * s[4];
  }
}

/* One hydro step of (rho, m, e) in place over dt; order 1 (cell-centred
 * states) or 2 (the van Leer step).  work: 36 N + 5 Nf doubles.  Returns 0,
 * or -1 if a state became unphysical (non-positive density or pressure). */
int orc_hydro_step(const orc_problem *p, double dt, int order, double *rho, double *m, double *e,
                   double *work) {
  const int64_t N = p->n_cells;
  double *W = work, *grad = W + 5 * N, *rh = grad + 15 * N, *mh = rh + N, *eh = mh + 3 * N;
  double *Fa = eh + N;  /* 5 Nf */
  for (int64_t c = 0; c < N; ++c) hydro_prim(p->gamma_gas, rho[c], m + 3 * c, e[c], W + 5 * c);
  if (order == 1) {
    if (hydro_face_fluxes(p, W, NULL, Fa) != 0) return -1;
    hydro_apply(p, dt, Fa, rho, m, e, rho, m, e);
  } else {
    /* half step with the cell-centred states */
    if (hydro_face_fluxes(p, W, NULL, Fa) != 0) return -1;
    hydro_apply(p, 0.5 * dt, Fa, rho, m, e, rh, mh, eh);
    for (int64_t c = 0; c < N; ++c) hydro_prim(p->gamma_gas, rh[c], mh + 3 * c, eh[c], W + 5 * c);
    for (int64_t c = 0; c < N; ++c)
      if (!(W[5 * c] > 0.0) || !(W[5 * c + 4] > 0.0)) return -1;
    /* limited least-squares gradients of the five primitives */
    orc_problem q = *p;
    q.n_angles = 5;
    orc_gradient(&q, W, 1, grad);
    if (hydro_face_fluxes(p, W, grad, Fa) != 0) return -1;
    hydro_apply(p, dt, Fa, rho, m, e, rho, m, e);
  }
  for (int64_t c = 0; c < N; ++c) {
    double Wc[5];
    hydro_prim(p->gamma_gas, rho[c], m + 3 * c, e[c], Wc);
    if (!(Wc[0] > 0.0) || !(Wc[4] > 0.0)) return -1;
  }
  return 0;
}
