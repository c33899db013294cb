"""The five synthetic workloads, shaped like the paper's test problems (Sec. 3).

Every workload is a jittered periodic Voronoi box (unit box, lattice spacing
h = 1/n, jitter U(-0.25, 0.25) h per axis, seed = workload number unless
given) with a level-symmetric angle set, in code units: a = 1, ideal gas
P = rho * R * T with R = k_B / (mu m_p) = 1 and gamma = 5/3, so that
e_internal = rho T / (gamma - 1).

  thermal    16^3, S6 (48), rho = 1, T = 1, E_r = 10 a T^4 isotropic,
             kappa_P = kappa_J = 1, kappa_s = 0, v = 0, cbar = c = 100,
             CFL 0.3, 100 steps (Sec. 3.1, thermal equilibrium).
  shadows    128^3, S8 (80), kappa_a = 1e-3 background with three opaque
             spheres (r = 0.08, kappa_a = 1e3), four isotropic emitter
             cells, absorbing boundary layers on all six sides, two
             collimated beams entering through the -y layer at +-30 deg,
             cbar = c = 1e3, 200 steps (Sec. 3.4 and 3.5).
  diffusion  100^3, S6, mesh and gas moving with v = w = (0.3, 0, 0),
             cell optical depth kappa_a h log-uniform in [10, 1000],
             kappa_s = kappa_a, Gaussian E_r (sigma = 0.05) on T = 1,
             cbar = c = 1e3, 300 steps (Sec. 3.3).
  adjoint    64^3, S6, log-normal kappa_a (Gaussian random field, sigma 1,
             correlation length 0.1), absorbing layers at +-x, one
             emitter, cbar = c = 1, 64 steps.
  waves      256^3, S8, rho = 1, T = 1, E_r = 1, cell optical depth 1,
             cbar = 100, c = 1e4, small sinusoidal perturbation of T and
             E_r along x, 50 steps (Sec. 3.6 with the hydro frozen).

Boundary cells (kind 1) relax to a per-direction I0 (Sec. 2.4); emitter
cells (kind 2) relax to I_src at rate cbar * emit_rate (Sec. 2.5).  I0 is
stored as a few shared rows; bc_row[c] selects the row of cell c.
"""
from dataclasses import dataclass, field

import numpy as np

from .angles import level_symmetric
from .mesh import Mesh, build_mesh

KIND_INTERIOR, KIND_BOUNDARY, KIND_EMITTER = 0, 1, 2


@dataclass
class Problem:
    name: str
    mesh: Mesh
    dirs: np.ndarray          # [A, 3]
    weights: np.ndarray       # [A]
    cbar: float
    c: float
    a_rad: float
    gamma_gas: float
    r_gas: float
    cfl: float
    n_steps: int
    rho: np.ndarray           # [N]
    e: np.ndarray             # [N] total gas energy density
    m: np.ndarray             # [N, 3] gas momentum density
    kappa_P: np.ndarray       # [N]
    kappa_J: np.ndarray       # [N]
    kappa_s: np.ndarray       # [N]
    kind: np.ndarray          # [N] uint8
    tau: np.ndarray           # [N] boundary relaxation time
    emit_rate: np.ndarray     # [N] rho * kappa of emitter cells
    I_src: np.ndarray         # [N] emitter target intensity
    bc_row: np.ndarray        # [N] int32 row of I0 (-1 if none)
    I0: np.ndarray            # [n_rows, A]
    J0: np.ndarray            # [N] initial intensity scale per cell
    q0: np.ndarray            # [A] initial angular profile (I = J0 x q0)
    extra: dict = field(default_factory=dict)
    integrator: int = 0       # 0 first-order upwind step, 1 van Leer with limited linear reconstruction
    boost: int = 0            # 1: the comoving transformation to all orders in v/c (Gamma with gamma)
    gcl: int = 0              # 1: cell volumes follow the face velocities (geometric conservation law)
    beta_P: float = 0.0       # kappa_P(T) = kappa_P (T / T_ref)^beta_P, at T^{n+1} (beta_P >= -3)
    beta_J: float = 0.0       # kappa_J(T) = kappa_J (T / T_ref)^beta_J, at T^n
    T_ref: float = 1.0
    n_groups: int = 1         # frequency groups (kappa arrays [N][n_groups], intensities [N][n_groups * A])
    group_w: np.ndarray = None  # [n_groups] group weights

    @property
    def n_cells(self):
        return self.mesh.n_cells

    @property
    def n_angles(self):
        return int(self.dirs.shape[0])

    def initial_intensity(self, dtype=np.float64):
        return np.ascontiguousarray(np.outer(self.J0, self.q0).astype(dtype))

    def cfl_dt(self):
        """dt = CFL * min_c V_c^(1/3) / (cbar + |w|) (Courant limit; the
        paper defers the formula to its hydro scheme, this is the reading
        used throughout)."""
        wmax = float(np.max(np.linalg.norm(self.mesh.face_w, axis=1))) if self.mesh.n_faces else 0.0
        return self.cfl * float(np.min(np.cbrt(self.mesh.cell_volume))) / (self.cbar + wmax)


def _gas(N, rho, T, v, gamma, r_gas):
    rho = np.full(N, rho, dtype=np.float64) if np.isscalar(rho) else np.asarray(rho, np.float64)
    T = np.full(N, T, dtype=np.float64) if np.isscalar(T) else np.asarray(T, np.float64)
    v = np.broadcast_to(np.asarray(v, np.float64), (N, 3))
    m = rho[:, None] * v
    e = rho * r_gas * T / (gamma - 1.0) + 0.5 * np.sum(m * m, axis=1) / rho
    return rho, e, np.ascontiguousarray(m)


def _blank_cells(N, A):
    return (np.zeros(N, np.uint8), np.zeros(N), np.zeros(N), np.zeros(N),
            np.full(N, -1, np.int32), np.zeros((1, A)))


def _boundary_layers(mesh, axes):
    """Cells in the outer one-cell lattice layer on the listed axes."""
    ix = mesh.lattice_index()
    mark = np.zeros(mesh.n_cells, bool)
    for ax in axes:
        mark |= (ix[ax] == 0) | (ix[ax] == mesh.n[ax] - 1)
    return mark


def thermal(n=16, seed=1, steps=100, order=6):
    mesh = build_mesh((n, n, n), seed=seed)
    dirs, w = level_symmetric(order)
    N, A = mesh.n_cells, dirs.shape[0]
    gamma, r_gas = 5.0 / 3.0, 1.0
    rho, e, m = _gas(N, 1.0, 1.0, (0, 0, 0), gamma, r_gas)
    kind, tau, emit, isrc, bc_row, I0 = _blank_cells(N, A)
    return Problem("thermal", mesh, dirs, w, 100.0, 100.0, 1.0, gamma, r_gas, 0.3, steps,
                   rho, e, m, np.ones(N), np.ones(N), np.zeros(N), kind, tau, emit, isrc,
                   bc_row, I0, np.full(N, 10.0 / (4 * np.pi)), np.ones(A))


def _nearest_ordinates(dirs, b):
    b = np.asarray(b, np.float64) / np.linalg.norm(b)
    s = dirs @ b
    return np.nonzero(s >= s.max() - 1e-12)[0]


def shadows(n=128, seed=2, steps=200, order=8):
    mesh = build_mesh((n, n, n), seed=seed)
    dirs, w = level_symmetric(order)
    N, A = mesh.n_cells, dirs.shape[0]
    h = 1.0 / n
    gamma, r_gas = 5.0 / 3.0, 1.0
    rng = np.random.default_rng(1000 + seed)
    T0 = 1e-2
    rho, e, m = _gas(N, 1.0, T0, (0, 0, 0), gamma, r_gas)
    kap = np.full(N, 1e-3)
    x = mesh.points
    # three opaque spheres: the first on beam 1's path beyond the crossing
    s30, c30 = 0.5, np.sqrt(3.0) / 2.0
    centres = [np.array([0.35 + 0.55 * s30 / c30, 0.55, 0.5])]
    r_s = 0.08
    while len(centres) < 3:
        p = rng.uniform(0.2, 0.8, 3)
        if all(np.linalg.norm(p - q) > 2.2 * r_s for q in centres):
            centres.append(p)
    for p in centres:
        kap[np.sum((x - p) ** 2, axis=1) < r_s ** 2] = 1e3
    kind, tau, emit, isrc, bc_row, _ = _blank_cells(N, A)
    bmask = _boundary_layers(mesh, (0, 1, 2))
    kind[bmask] = KIND_BOUNDARY
    I0 = np.zeros((3, A))
    bc_row[bmask] = 0
    # beams: -y layer, discs of radius 0.05 in (x, z) around x = 0.35 / 0.65
    iy = mesh.lattice_index()[1]
    for k, (x0, bdir) in enumerate(((0.35, (s30, c30, 0.0)), (0.65, (-s30, c30, 0.0)))):
        sel = _nearest_ordinates(dirs, bdir)
        I0[k + 1, sel] = 10.0
        disc = (iy == 0) & ((x[:, 0] - x0) ** 2 + (x[:, 2] - 0.5) ** 2 < 0.05 ** 2)
        bc_row[disc] = k + 1
    # four isotropic emitters (one cell each) in the interior
    emitters = []
    while len(emitters) < 4:
        p = rng.uniform(0.1, 0.9, 3)
        c = int(np.argmin(np.sum((x - p) ** 2, axis=1)))
        if kind[c] == KIND_INTERIOR and c not in emitters:
            emitters.append(c)
    kind[emitters] = KIND_EMITTER
    emit[emitters] = 1.0 / h
    isrc[emitters] = 1.0
    J0 = np.full(N, T0 ** 4 / (4 * np.pi))
    prob = Problem("shadows", mesh, dirs, w, 1e3, 1e3, 1.0, gamma, r_gas, 0.3, steps,
                   rho, e, m, kap.copy(), kap.copy(), np.zeros(N), kind, tau, emit, isrc,
                   bc_row, I0, J0, np.ones(A))
    prob.extra.update(spheres=np.array(centres), sphere_r=r_s, emitters=np.array(emitters))
    return prob


def diffusion(n=100, seed=3, steps=300, order=6, v=(0.3, 0.0, 0.0)):
    mesh = build_mesh((n, n, n), seed=seed)
    mesh.face_w = np.ascontiguousarray(np.broadcast_to(np.asarray(v, np.float64), (mesh.n_faces, 3)))
    dirs, w = level_symmetric(order)
    N, A = mesh.n_cells, dirs.shape[0]
    h = 1.0 / n
    gamma, r_gas = 5.0 / 3.0, 1.0
    rng = np.random.default_rng(1000 + seed)
    rho, e, m = _gas(N, 1.0, 1.0, v, gamma, r_gas)
    tau_cell = np.exp(rng.uniform(np.log(10.0), np.log(1000.0), N))
    kap = tau_cell / h
    r2 = np.sum((mesh.points - 0.5) ** 2, axis=1)
    sigma = 0.05
    E = 1.0 + 10.0 * np.exp(-r2 / (2 * sigma ** 2))
    c = 1e3
    gam = 1.0 - dirs @ np.asarray(v, np.float64) / c
    kind, tau, emit, isrc, bc_row, I0 = _blank_cells(N, A)
    # comoving-isotropic radiation: lab I_a = (E / 4 pi) / Gamma_a^4
    return Problem("diffusion", mesh, dirs, w, 1e3, c, 1.0, gamma, r_gas, 0.3, steps,
                   rho, e, m, kap.copy(), kap.copy(), kap.copy(), kind, tau, emit, isrc,
                   bc_row, I0, E / (4 * np.pi), 1.0 / gam ** 4)


def gaussian_random_field(n, corr, seed):
    """Zero-mean unit-variance field on an n^3 periodic lattice (unit box)
    with Gaussian correlation exp(-r^2 / corr^2), by FFT filtering."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n, n, n))
    k = 2 * np.pi * np.fft.fftfreq(n, d=1.0 / n)
    kx, ky, kz = np.meshgrid(k, k, k, indexing="ij")
    filt = np.exp(-(kx ** 2 + ky ** 2 + kz ** 2) * corr ** 2 / 8.0)
    g = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    g -= g.mean()
    return g / g.std()


def adjoint(n=64, seed=4, steps=64, order=6):
    mesh = build_mesh((n, n, n), seed=seed)
    dirs, w = level_symmetric(order)
    N, A = mesh.n_cells, dirs.shape[0]
    gamma, r_gas = 5.0 / 3.0, 1.0
    rho, e, m = _gas(N, 1.0, 1.0, (0, 0, 0), gamma, r_gas)
    g = gaussian_random_field(n, 0.1, 1000 + seed).ravel()
    kap = np.exp(g)
    kind, tau, emit, isrc, bc_row, I0 = _blank_cells(N, A)
    bmask = _boundary_layers(mesh, (0,))
    kind[bmask] = KIND_BOUNDARY
    bc_row[bmask] = 0
    c = int(np.argmin(np.sum((mesh.points - np.array([0.85, 0.5, 0.5])) ** 2, axis=1)))
    kind[c] = KIND_EMITTER
    emit[c] = float(n)
    isrc[c] = 1.0
    prob = Problem("adjoint", mesh, dirs, w, 1.0, 1.0, 1.0, gamma, r_gas, 0.3, steps,
                   rho, e, m, kap.copy(), kap.copy(), np.zeros(N), kind, tau, emit, isrc,
                   bc_row, I0, np.full(N, 1.0 / (4 * np.pi)), np.ones(A))
    prob.extra.update(emitter=c, checkpoint_every=8)
    return prob


def waves(n=256, seed=5, steps=50, order=8, amplitude=1e-6):
    mesh = build_mesh((n, n, n), seed=seed)
    dirs, w = level_symmetric(order)
    N, A = mesh.n_cells, dirs.shape[0]
    gamma, r_gas = 5.0 / 3.0, 1.0
    kx = 2 * np.pi * mesh.points[:, 0]
    T = 1.0 + amplitude * np.sin(kx)
    rho, e, m = _gas(N, 1.0, T, (0, 0, 0), gamma, r_gas)
    kap = np.full(N, float(n))
    kind, tau, emit, isrc, bc_row, I0 = _blank_cells(N, A)
    J0 = (1.0 + 4.0 * amplitude * np.sin(kx)) / (4 * np.pi)
    return Problem("waves", mesh, dirs, w, 100.0, 1e4, 1.0, gamma, r_gas, 0.3, steps,
                   rho, e, m, kap.copy(), kap.copy(), np.zeros(N), kind, tau, emit, isrc,
                   bc_row, I0, J0, np.ones(A))


WORKLOADS = {"thermal": thermal, "shadows": shadows, "diffusion": diffusion,
             "adjoint": adjoint, "waves": waves}


def make_problem(name, **kw) -> Problem:
    return WORKLOADS[name](**kw)
