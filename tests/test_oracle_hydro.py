"""CPU pins of the oracle's hydrodynamics and of radiation subcycled under
it (Sec. 2: Eq. time evolution with the Euler fluxes, the HLLC Riemann
solver in the face frame and the van Leer step; Sec. 3.6: the radiative
linear wave).

Each test checks the oracle against something other than itself:
* the HLLC flux of equal states is the physical flux, the flux seen from the
  other side of a face is its negative, and a stationary contact passes no
  mass or energy (the solver's defining property, Toro Sec. 10.4);
* the Sod shock tube converges to the exact Riemann solution, written out
  here from the textbook pressure function (Toro Ch. 4);
* mass, momentum and energy are conserved to rounding, and a uniform moving
  gas stays uniform, on a jittered periodic mesh;
* a small-amplitude sound wave converges at second order (the paper reports
  -1.74 for its moving-mesh solver, Sec. 3.6; the van Leer step with limited
  linear reconstruction is formally second order);
* the radiation-modified linear wave of Sec. 3.6 (c/c_s = 1.45e3,
  cbar/c = 1e-2, P_rad = P_gas) converges, at first order or better, to the
  mode of the radiation-hydrodynamics equations linearised about rest, whose
  eigenvalue numpy computes from the equations written out here.
"""
import numpy as np
import pytest

import oracle
from paper_2002_08377_gb300.inputs import Problem, build_mesh, level_symmetric


@pytest.fixture(autouse=True)
def _one_thread():
    # these meshes have a few hundred cells: one thread avoids the OpenMP
    # overhead of many small loops
    n = oracle.set_threads(0)
    oracle.set_threads(1)
    yield
    oracle.set_threads(n)


def gas_problem(mesh, rho, v, P, gamma, dirs=None, w=None, a_rad=0.0, cbar=1.0, c=1.0, kappa=0.0,
                I=None, r_gas=1.0):
    """A problem record for a gas state (rho, v [N][3], P) on mesh; with
    kappa = 0 and a_rad = 0 the radiation is inert."""
    if dirs is None:
        dirs, w = level_symmetric(2)
    N, A = mesh.n_cells, dirs.shape[0]
    m = rho[:, None] * v
    e = P / (gamma - 1.0) + 0.5 * rho * np.sum(v * v, axis=1)
    k = np.full(N, float(kappa))
    z = np.zeros(N)
    prob = Problem("gas", mesh, dirs, w, cbar, c, a_rad, gamma, r_gas, 0.3, 0, rho.copy(), e, m,
                   k.copy(), k.copy(), z.copy(), np.zeros(N, np.uint8), z.copy(), z.copy(), z.copy(),
                   np.full(N, -1, np.int32), np.zeros((1, A)), np.ones(N), np.zeros(A))
    if I is not None:
        prob.initial_intensity = lambda dtype=np.float64, _I=I: np.ascontiguousarray(_I.astype(dtype))
    return prob


def quasi_1d(N, jitter, seed=1):
    """N x 2 x 2 periodic cells of side 1/N (box 1 x 2/N x 2/N)."""
    return build_mesh((N, 2, 2), box=(1.0, 2.0 / N, 2.0 / N), jitter=jitter, seed=seed)


# ------------------------------------------------------------------ HLLC
def _physical_flux(W, n, g):
    rho, v, P = W[0], np.asarray(W[1:4]), W[4]
    u = v @ n
    E = P / (g - 1) + 0.5 * rho * v @ v
    return np.concatenate([[rho * u], rho * v * u + P * np.asarray(n), [(E + P) * u]])


def test_hllc_consistency_symmetry_and_contact():
    rng = np.random.default_rng(0)
    g = 5.0 / 3.0
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        WL = np.concatenate([[rng.uniform(0.1, 3)], rng.normal(size=3), [rng.uniform(0.1, 3)]])
        WR = np.concatenate([[rng.uniform(0.1, 3)], rng.normal(size=3), [rng.uniform(0.1, 3)]])
        F = oracle.hllc_flux(g, WL, WL, n)
        ref = _physical_flux(WL, n, g)
        assert np.abs(F - ref).max() <= 1e-14 * np.abs(ref).max() * 10
        F1 = oracle.hllc_flux(g, WL, WR, n)
        F2 = oracle.hllc_flux(g, WR, WL, -n)
        assert np.abs(F1 + F2).max() <= 1e-13 * np.abs(F1).max()
    # a stationary contact: density jump, equal pressure, no velocity
    n = np.array([0.6, 0.0, 0.8])
    F = oracle.hllc_flux(g, [1.0, 0, 0, 0, 1.0], [0.125, 0, 0, 0, 1.0], n)
    assert F[0] == 0.0 and F[4] == 0.0
    assert np.array_equal(F[1:4], 1.0 * n)


# ------------------------------------------------------------------ Riemann problem
def exact_riemann(L, R, g, xi):
    """Exact solution (rho, u, p) of the 1-D Riemann problem with left and
    right states (rho, u, p) at the similarity coordinate xi = x / t: the
    star pressure is the root of f_L(p) + f_R(p) + u_R - u_L = 0 (shock or
    rarefaction branch of each side), then the wave pattern is sampled."""
    from scipy.optimize import brentq
    rl, ul, pl = L
    rr, ur, pr = R
    al, ar = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)

    def f(p, rk, pk, ak):
        if p > pk:
            A, B = 2 / ((g + 1) * rk), (g - 1) / (g + 1) * pk
            return (p - pk) * np.sqrt(A / (p + B))
        return 2 * ak / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)

    ps = brentq(lambda p: f(p, rl, pl, al) + f(p, rr, pr, ar) + ur - ul, 1e-12, 100 * max(pl, pr))
    us = 0.5 * (ul + ur) + 0.5 * (f(ps, rr, pr, ar) - f(ps, rl, pl, al))
    gm = (g - 1) / (g + 1)
    out = np.empty((len(xi), 3))
    for i, x in enumerate(xi):
        # mirror the right side onto the left one
        left = x <= us
        rk, uk, pk, ak, s = (rl, ul, pl, al, 1.0) if left else (rr, -ur, pr, ar, -1.0)
        xx, u_s = s * x, s * us
        if ps > pk:  # shock
            S = uk - ak * np.sqrt((g + 1) / (2 * g) * ps / pk + (g - 1) / (2 * g))
            state = (rk, uk, pk) if xx <= S else (rk * (ps / pk + gm) / (gm * ps / pk + 1), u_s, ps)
        else:  # rarefaction
            head, tail = uk - ak, u_s - ak * (ps / pk) ** ((g - 1) / (2 * g))
            if xx <= head:
                state = (rk, uk, pk)
            elif xx >= tail:
                state = (rk * (ps / pk) ** (1 / g), u_s, ps)
            else:
                u = 2 / (g + 1) * (ak + (g - 1) / 2 * uk + xx)
                a = 2 / (g + 1) * (ak + (g - 1) / 2 * (uk - xx))
                state = (rk * (a / ak) ** (2 / (g - 1)), u, pk * (a / ak) ** (2 * g / (g - 1)))
        out[i] = (state[0], s * state[1], state[2])
    return out


def _sod_error(N, jitter, tend=0.1):
    g = 1.4
    mesh = quasi_1d(N, jitter, seed=2)
    x = mesh.cell_centroid[:, 0] % 1.0
    hi = (x >= 0.25) & (x < 0.75)
    rho = np.where(hi, 1.0, 0.125)
    P = np.where(hi, 1.0, 0.1)
    o = oracle.Oracle(gas_problem(mesh, rho, np.zeros((mesh.n_cells, 3)), P, g))
    t = 0.0
    while t < tend - 1e-15:
        dt = min(o.hydro_dt(0.3), tend - t)
        o.hydro_step(dt)
        t += dt
    # Sod's problem at x = 0.75 (high state on the left) and its mirror image at 0.25
    sod = exact_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g, (np.abs(x - 0.5) - 0.25) / tend)
    V = mesh.cell_volume
    return np.sum(V * np.abs(o.rho - sod[:, 0])) / np.sum(V)


@pytest.mark.parametrize("jitter", [0.0, 0.1])
def test_sod_shock_tube_converges_to_exact_solution(jitter):
    """The density's L1 error against the exact Riemann solution falls at
    about first order (the order a discontinuous solution allows)."""
    errs = np.array([_sod_error(N, jitter) for N in (64, 128, 256)])
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders > 0.75), (errs, orders)
    assert errs[-1] < 5e-3, errs


# ------------------------------------------------------------------ invariants
def test_conservation_and_free_stream():
    """Jittered periodic mesh: a smooth random state conserves mass,
    momentum and energy to rounding over 20 steps (both orders), and a
    uniform moving gas stays uniform to rounding."""
    mesh = build_mesh((6, 5, 4), jitter=0.25, seed=3)
    rng = np.random.default_rng(1)
    N = mesh.n_cells
    x = mesh.cell_centroid
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])
    v = 0.3 * rng.normal(size=(N, 3))
    P = 1.0 + 0.2 * np.cos(2 * np.pi * x[:, 2])
    V = mesh.cell_volume
    for order in (1, 2):
        o = oracle.Oracle(gas_problem(mesh, rho, v, P, 5.0 / 3.0))
        tot0 = np.array([V @ o.rho, *(V @ o.m), V @ o.e])
        for _ in range(20):
            o.hydro_step(o.hydro_dt(0.3), order)
        tot1 = np.array([V @ o.rho, *(V @ o.m), V @ o.e])
        assert np.abs(tot1 - tot0).max() <= 1e-14 * np.abs(tot0).max() * 10
    u = np.broadcast_to([0.4, -0.3, 0.2], (N, 3))
    o = oracle.Oracle(gas_problem(mesh, np.full(N, 1.3), u.copy(), np.full(N, 0.7), 5.0 / 3.0))
    for _ in range(10):
        o.hydro_step(o.hydro_dt(0.3))
    assert np.abs(o.rho / 1.3 - 1).max() < 1e-13
    assert np.abs(o.m / (1.3 * u) - 1).max() < 1e-12


# ------------------------------------------------------------------ sound wave
def _acoustic_error(N, jitter, amp=1e-6):
    g = 5.0 / 3.0
    mesh = quasi_1d(N, jitter)
    cs, k = np.sqrt(g), 2 * np.pi
    s = np.sin(k * mesh.cell_centroid[:, 0])
    rho = 1.0 + amp * s
    v = np.zeros((mesh.n_cells, 3))
    v[:, 0] = cs * amp * s
    o = oracle.Oracle(gas_problem(mesh, rho, v, 1.0 + g * amp * s, g))
    t, T = 0.0, 1.0 / cs  # one period of the wave
    while t < T - 1e-15:
        dt = min(o.hydro_dt(0.3), T - t)
        o.hydro_step(dt)
        t += dt
    V = mesh.cell_volume
    return np.sum(V * np.abs(o.rho - rho)) / np.sum(V) / amp


@pytest.mark.parametrize("jitter", [0.0, 0.1])
def test_acoustic_wave_converges_at_second_order(jitter):
    """After one period the wave's L1 error falls at second order, at least
    the paper's -1.74, on a lattice and with 10 % jitter (Sec. 3.6)."""
    errs = np.array([_acoustic_error(N, jitter) for N in (16, 32, 64, 128)])
    slope = np.polyfit(np.log([16, 32, 64, 128]), np.log(errs), 1)[0]
    assert slope <= -1.74, (errs, slope)


# ------------------------------------------------------------------ radiative linear wave
def radhydro_linear_system(dirs, w, k, g, rho0, T0, r_gas, a, c, cbar, kap):
    """Radiation hydrodynamics linearised about rest (v = 0, rho0, T0,
    isotropic I0 = a T0^4 / 4 pi) for perturbations exp(i k x) along x, first
    order in v/c, kappa_P = kappa_J = kap per unit mass, no scattering
    (Eq. time evolution with the Euler fluxes; Eqs. com radiative source,
    gas1, gas2 in their continuous form): with B0 = a T0^4 / 4 pi,
      d rho/dt = -i k rho0 dv,
      d v/dt   = -i k (r / rho0)(rho0 dT + T0 drho) + 4 pi kap sum w n_x dI
                 - (16 pi B0 kap / 3c) dv,
      d T/dt   = -i k (gamma - 1) T0 dv - (4 pi c kap / c_v)(4 B0 dT / T0 - sum w dI),
      d I_a/dt = -i k cbar n_ax dI_a + cbar rho0 kap (4 B0 dT / T0 - dI_a + 4 B0 n_ax dv / c).
    Returns the matrix of d/dt acting on (drho, dv, dT, dI_1 .. dI_A)."""
    A = len(w)
    cv = r_gas / (g - 1)
    B0 = a * T0 ** 4 / (4 * np.pi)
    M = np.zeros((A + 3, A + 3), complex)
    M[0, 1] = -1j * k * rho0
    M[1, 0] = -1j * k * r_gas * T0 / rho0
    M[1, 2] = -1j * k * r_gas
    M[1, 1] = -16 * np.pi * B0 * kap / (3 * c)
    M[1, 3:] = 4 * np.pi * kap * w * dirs[:, 0]
    M[2, 1] = -1j * k * (g - 1) * T0
    M[2, 2] = -(4 * np.pi * c * kap / cv) * 4 * B0 / T0
    M[2, 3:] = (4 * np.pi * c * kap / cv) * w
    M[3 + np.arange(A), 3 + np.arange(A)] = -1j * k * cbar * dirs[:, 0] - cbar * rho0 * kap
    M[3:, 2] = cbar * rho0 * kap * 4 * B0 / T0
    M[3:, 1] = cbar * rho0 * kap * 4 * B0 * dirs[:, 0] / c
    return M


def radwave_problem(N, tau, amp=1e-6, jitter=0.1, C=1.45e3):
    """The Sec. 3.6 setup in code units: rho0 = T0 = r_gas = 1 (isothermal
    sound speed 1), c = 1.45e3, cbar = c / 100, a = 3 (P_rad = P_gas),
    kappa = tau (optical depth tau over the wavelength, the box length 1),
    S2 directions, lattice jitter 10 %, with the right-running sound mode of
    the linear system laid on the mesh at amplitude amp.  Returns (problem,
    mode eigenvalue, its vector).  C = c / c_s (1.45e3 in the paper)."""
    g, rho0, T0, r = 5.0 / 3.0, 1.0, 1.0, 1.0
    c = C  # c / c_s with the isothermal sound speed 1
    cbar, a, kap, k = 1e-2 * c, 3.0, tau, 2 * np.pi
    dirs, w = level_symmetric(2)
    M = radhydro_linear_system(dirs, w, k, g, rho0, T0, r, a, c, cbar, kap)
    lam, vec = np.linalg.eig(M)
    # the mode with a density part whose phase speed is closest to the
    # adiabatic sound speed, running towards +x
    cand = [i for i in range(len(lam)) if lam[i].imag < 0 and abs(vec[0, i]) > 1e-6 * np.abs(vec[:, i]).max()]
    i = min(cand, key=lambda i: abs(-lam[i].imag / k - np.sqrt(g)))
    X = vec[:, i] / vec[0, i]
    mesh = quasi_1d(N, jitter)
    ph = np.exp(1j * k * mesh.cell_centroid[:, 0])
    part = lambda z: amp * np.real(z * ph)
    rho, T = rho0 + part(X[0]), T0 + part(X[2])
    v = np.zeros((mesh.n_cells, 3))
    v[:, 0] = part(X[1])
    I = a * T0 ** 4 / (4 * np.pi) + amp * np.real(X[3:][None, :] * ph[:, None])
    prob = gas_problem(mesh, rho, v, rho * r * T, g, dirs, w, a, cbar, c, kap, I, r)
    return prob, lam[i], X


def radwave(N, tau, amp=1e-6, jitter=0.1):
    """radwave_problem run on the oracle for one isothermal sound crossing
    time (t = 1), the radiation subcycled under each hydro step (as many
    Courant steps of the radiation as fit in the gas's Courant step).
    Returns (problem, mode eigenvalue, its vector, the oracle after the run,
    end time)."""
    prob, lam, X = radwave_problem(N, tau, amp, jitter)
    o = oracle.Oracle(prob)
    t_end = 1.0
    dt_rad = o.cfl_dt()
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(o.hydro_dt(0.3), t_end - t)
        assert o.radhydro_step(dt, int(np.ceil(dt / dt_rad))) == oracle.ORC_OK
        t += dt
    return prob, lam, X, o, t_end


def _radwave_error(N, tau):
    prob, lam, X, o, t_end = radwave(N, tau)
    mesh = prob.mesh
    ph = np.exp(1j * 2 * np.pi * mesh.cell_centroid[:, 0])
    V = mesh.cell_volume
    c0 = np.sum(V * (prob.rho - 1.0) * np.conj(ph))
    c1 = np.sum(V * (o.rho - 1.0) * np.conj(ph))
    pred = np.exp(lam * t_end)
    return abs(c1 / c0 - pred) / abs(pred)


@pytest.mark.parametrize("tau", [0.01, 1.0, 100.0])
def test_radiative_linear_wave_converges_to_dispersion_relation(tau):
    """The density mode's complex amplitude after one sound crossing (its
    damping and phase) converges at first order or better in the cell size
    to exp(lambda t) of the linear system (Sec. 3.6 reports first order)."""
    errs = np.array([_radwave_error(N, tau) for N in (16, 32, 64)])
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders > 0.8), (errs, orders)
    assert errs[-1] < 0.05, errs
