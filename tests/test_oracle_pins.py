"""CPU pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a textbook scheme, an invariant, brute force, or the paper's own
worked example.  None of these calls the CUDA path.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2002_08377_gb300.inputs import build_mesh, level_symmetric, thermal
from tests._problems import make, randomise

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- mesh, angles
def _closure(M):
    S = np.zeros((M.n_cells, 3))
    av = M.face_area[:, None] * M.face_normal
    np.add.at(S, M.face_cells[:, 0], av)
    np.add.at(S, M.face_cells[:, 1], -av)
    return S


@pytest.mark.parametrize("n", [(2, 2, 2), (4, 3, 5), (10, 10, 10)])
def test_mesh_geometry_invariants(n):
    """Closed cells (sum_f A n = 0), volumes tile the box, and the
    divergence theorem sum_f A (r_f - x).n = 3V (Sec. 2, Gauss' theorem)."""
    M = build_mesh(n, jitter=0.25, seed=3)
    assert abs(M.cell_volume.sum() - 1.0) < 1e-13
    assert np.abs(_closure(M)).max() < 1e-13 * M.face_area.mean() * 10
    div = np.zeros(M.n_cells)
    i, j = M.face_cells[:, 0], M.face_cells[:, 1]
    shift = M.face_shift * M.box
    div += np.bincount(i, M.face_area * np.einsum("ij,ij->i", M.face_centroid - M.points[i],
                                                     M.face_normal), M.n_cells)
    div -= np.bincount(j, M.face_area * np.einsum("ij,ij->i", M.face_centroid - shift - M.points[j],
                                                     M.face_normal), M.n_cells)
    assert np.abs(div - 3 * M.cell_volume).max() < 1e-12 * M.cell_volume.mean()


def test_mesh_against_qhull():
    """Cell volumes agree with scipy's Qhull on periodic replicas."""
    spatial = pytest.importorskip("scipy.spatial")
    M = build_mesh((4, 4, 4), jitter=0.25, seed=5)
    pts = M.points
    reps = []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                reps.append(pts + np.array([dx, dy, dz], float))
    allp = np.concatenate(reps)
    vor = spatial.Voronoi(allp)
    centre = 13 * M.n_cells  # (0,0,0) replica block
    for c in range(M.n_cells):
        reg = vor.regions[vor.point_region[centre + c]]
        assert -1 not in reg
        hull = spatial.ConvexHull(vor.vertices[reg])
        assert abs(hull.volume - M.cell_volume[c]) < 1e-10


def test_cubic_lattice_is_exact():
    M = build_mesh((4, 5, 6), jitter=0.0)
    assert M.n_faces == 3 * M.n_cells
    assert np.allclose(M.cell_volume, 1.0 / 120.0, rtol=1e-14)


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_angle_set_moments(order):
    d, w = level_symmetric(order)
    A = order * (order + 2)
    assert d.shape == (A, 3)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    assert np.abs(w @ d).max() < 1e-15
    assert np.allclose(np.einsum("a,ai,aj->ij", w, d, d), np.eye(3) / 3, atol=1e-15)
    assert np.array_equal(d[A // 2:], -d[: A // 2])  # antipode of a is a + A/2


# ---------------------------------------------------------------- quartic (P10)
def test_newton_matches_mpmath_root():
    """Newton root of alpha T^4 + beta T = g within 4 ulp of a 60-digit
    bisection, over 30 decades of coefficients."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    rng = np.random.default_rng(0)
    for _ in range(400):
        a, b, g = 10.0 ** rng.uniform(-15, 15, 3)
        st, T, it = oracle.newton(a, b, g)
        assert st == 0 and it <= 64
        A, B, G = mp.mpf(a), mp.mpf(b), mp.mpf(g)
        lo, hi = mp.mpf(0), min(G / B, (G / A) ** mp.mpf(0.25))
        for _k in range(220):
            mid = (lo + hi) / 2
            if A * mid ** 4 + B * mid - G > 0:
                hi = mid
            else:
                lo = mid
        ref = float((lo + hi) / 2)
        assert abs(T - ref) <= 4 * np.spacing(ref), (a, b, g, T, ref)


def test_ferrari_cross_check():
    """The closed-form (Ferrari) root agrees with Newton where the quartic is
    well conditioned (neither term negligible)."""
    rng = np.random.default_rng(1)
    for _ in range(2000):
        T = 10.0 ** rng.uniform(-3, 3)
        a = 10.0 ** rng.uniform(-6, 6)
        b = a * T ** 3 * 10.0 ** rng.uniform(-2, 2)
        g = a * T ** 4 + b * T
        st, Tn, _ = oracle.newton(a, b, g)
        assert st == 0
        assert abs(Tn - T) <= 8 * np.spacing(T)
        assert abs(oracle.ferrari(a, b, g) - T) <= 1e-8 * T


def test_newton_reports_nonconvergence():
    st, T, it = oracle.newton(1.0, 1e6, 2e8, max_iter=1)  # root T = 100, start 119
    assert st == oracle.ORC_ERR_NONCONV and it == 1


# ---------------------------------------------------------------- transport
@pytest.mark.parametrize("w", [None, (0.3, -0.2, 0.1)])
def test_transport_is_donor_cell_on_cubic_lattice(w):
    """On an unjittered lattice the Voronoi faces are the cube faces and the
    upwind flux of Sec. 2.2 is the textbook donor-cell scheme."""
    n = (5, 4, 6)
    prob = make(n=n, order=4, jitter=0.0, w=w, cbar=2.0)
    rng = np.random.default_rng(2)
    I = rng.uniform(0, 1, (prob.n_cells, prob.n_angles))
    o = oracle.Oracle(prob)
    dt = 0.01
    out = o.transport(dt, I)
    h = 1.0 / np.array(n, float)
    wv = np.zeros(3) if w is None else np.asarray(w, float)
    for a in range(prob.n_angles):
        f = I[:, a].reshape(n)
        ref = f.copy()
        for d in range(3):
            s = prob.cbar * prob.dirs[a, d] - wv[d]
            if s > 0:
                ref -= dt * s / h[d] * (f - np.roll(f, 1, axis=d))
            elif s < 0:
                ref -= dt * s / h[d] * (np.roll(f, -1, axis=d) - f)
        assert np.allclose(out[:, a], ref.ravel(), rtol=1e-13, atol=1e-15)


def test_transport_invariants_jittered():
    """Uniform fields are preserved, sum_c V_c I_ca is conserved, and the
    update is positive and bounded (max principle) for dt <= 1/K."""
    prob = make(n=(6, 5, 4), order=6, w=(0.5, 0.0, -0.3), cbar=3.0)
    o = oracle.Oracle(prob)
    dt = 1.0 / o.positivity()
    rng = np.random.default_rng(3)
    U = np.full((prob.n_cells, prob.n_angles), 0.7)
    assert np.abs(o.transport(dt, U) - 0.7).max() < 1e-13
    I = rng.uniform(0, 1, U.shape)
    out = o.transport(dt, I)
    V = prob.mesh.cell_volume
    assert np.allclose(V @ out, V @ I, rtol=1e-13)
    assert out.min() >= -1e-14 and out.max() <= I.max() + 1e-14
    # closed form of the positivity bound on a cube lattice: K = cbar sum_d |n_d| / h_d
    prob2 = make(n=(4, 4, 4), order=6, jitter=0.0, cbar=3.0)
    K = oracle.Oracle(prob2).positivity()
    assert abs(K - 3.0 * 4 * np.abs(prob2.dirs).sum(1).max()) < 1e-12 * K


def test_crossing_beams_superpose():
    """Sec. 3.4: with no opacity and no motion the source step is the
    identity, so each ordinate is transported independently: a beam's
    channel is bit-identical with and without the other beam."""
    from paper_2002_08377_gb300.inputs import shadows
    base = shadows(n=12, steps=20)
    N = base.n_cells
    for k in ("kappa_P", "kappa_J", "kappa_s"):
        setattr(base, k, np.zeros(N))
    base.kind[base.kind == 2] = 0
    base.emit_rate[:] = 0
    rows = base.I0.copy()
    chan = [np.nonzero(rows[1])[0], np.nonzero(rows[2])[0]]

    def run(keep):
        base.I0 = rows.copy()
        for k in (1, 2):
            if k not in keep:
                base.I0[k] = 0.0
        o = oracle.Oracle(base)
        dt = o.cfl_dt()
        assert o.run(20, dt) == 0
        return o.I

    both, one, two = run((1, 2)), run((1,)), run((2,))
    assert np.array_equal(both[:, chan[0]], one[:, chan[0]])
    assert np.array_equal(both[:, chan[1]], two[:, chan[1]])
    assert one[:, chan[0]].max() > 1.0  # the beam entered the box


# ---------------------------------------------------------------- source (P1, P2, P4)
def _scalar_recurrence(steps, dt, rho, kP, kJ, T, J, cbar, c, a, rcv, mp):
    """Sec. 2.3 for an isotropic field at rest: the per-angle update collapses
    to J' = (J + x_P B(T')) / (1 + x_J), rho c_v (T' - T) = dt c rho (4 pi kJ
    J' - kP a T'^4); each step is solved with mpmath's root finder."""
    out = []
    xP, xJ = dt * cbar * rho * kP, dt * cbar * rho * kJ
    for _ in range(steps):
        def f(Tn, J=J, T=T):
            Jn = (J + xP * a * Tn ** 4 / (4 * mp.pi)) / (1 + xJ)
            return rcv * (Tn - T) - dt * c * rho * (4 * mp.pi * kJ * Jn - kP * a * Tn ** 4)
        Tn = mp.findroot(f, T)
        J = (J + xP * a * Tn ** 4 / (4 * mp.pi)) / (1 + xJ)
        T = Tn
        out.append((T, J))
    return out


@pytest.mark.parametrize("kS", [0.0, 3.0])
def test_thermal_relaxation_matches_scalar_recurrence(kS):
    """Uniform medium (the thermal equilibrium test, Sec. 3.1): the oracle's
    cells follow the scalar recurrence to 1e-12; isotropic scattering has no
    effect on an isotropic field at rest."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    prob = make(n=(4, 4, 4), order=6, cbar=100.0, c=100.0, kP=1.0, kJ=2.0, kS=kS,
                J0=10.0 / (4 * np.pi))
    o = oracle.Oracle(prob)
    dt = o.cfl_dt()
    ref = _scalar_recurrence(30, mp.mpf(dt), 1, 1, 2, mp.mpf(1), mp.mpf(10) / (4 * mp.pi),
                             mp.mpf(100), mp.mpf(100), 1, mp.mpf(1.5), mp)
    for s in range(30):
        assert o.step(dt) == 0
        T_ref, J_ref = float(ref[s][0]), float(ref[s][1])
        assert np.abs(o.temperature() / T_ref - 1).max() < 1e-12
        assert np.abs(o.I / J_ref - 1).max() < 1e-12


def test_thermal_workload_equilibrium_and_ode_order():
    """The thermal workload reaches the equilibrium of 1.5 T + T^4 = 11.5
    (energy balance with E_r = 10 a T^4 initially, c = cbar), and the
    implicit scheme converges at first order to the ODE
    dJ/dt = cbar rho (kP a T^4/4pi - kJ J), rho c_v dT/dt = c rho (4 pi kJ J - kP a T^4)."""
    from scipy.integrate import solve_ivp
    from scipy.optimize import brentq
    T_eq = brentq(lambda T: 1.5 * T + T ** 4 - 11.5, 0.5, 3.0)
    prob = thermal(n=6, steps=100)
    o = oracle.Oracle(prob)
    dt = o.cfl_dt()
    assert o.run(2000, dt) == 0
    assert np.abs(o.temperature() - T_eq).max() < 1e-10

    def rhs(t, y):
        J, T = y
        return [100.0 * (T ** 4 / (4 * np.pi) - J), 100.0 / 1.5 * (4 * np.pi * J - T ** 4)]

    t_end = 0.004
    sol = solve_ivp(rhs, (0, t_end), [10 / (4 * np.pi), 1.0], rtol=1e-12, atol=1e-14)
    errs = []
    for k in (40, 80, 160):
        o = oracle.Oracle(thermal(n=4))
        assert o.run(k, t_end / k) == 0
        errs.append(abs(o.temperature().mean() - sol.y[1, -1]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.8 < r1 < 2.2 and 1.8 < r2 < 2.2


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_paper_worked_example_equilibrium_temperature():
    """Sec. 3.1: atomic hydrogen at rho = 1e-15 g/cc, T_gas = 10 K, radiation
    at 200 K, cbar = c, equilibrates at 101.7 K (printed value).  CGS
    constants (mu = 1, gamma = 5/3, m_p) give 101.33 K from the energy
    balance; the paper's constants are unstated, so the printed value is
    held to 0.5 % and our energy balance exactly."""
    from scipy.optimize import brentq
    g = _read_golden("thermal_equilibrium_cgs.txt")
    kB, mp_, a, c = 1.380649e-16, 1.67262192e-24, 7.565733e-15, 2.99792458e10
    rcv = g["rho"] * kB / (mp_ * (5.0 / 3.0 - 1.0))
    E0 = rcv * g["T_gas"] + a * g["T_rad"] ** 4
    T_bal = brentq(lambda T: rcv * T + a * T ** 4 - E0, 1.0, 1e3)
    for kappa in (g["kappa_1"], g["kappa_2"]):
        prob = make(n=(2, 2, 2), order=2, cbar=c, c=c, a_rad=a, r_gas=kB / mp_, rho=g["rho"],
                    T=g["T_gas"], kP=kappa, kJ=kappa, J0=a * g["T_rad"] ** 4 / (4 * np.pi))
        o = oracle.Oracle(prob)
        dt = 1e9  # seconds; the implicit source is stable far beyond the thermal time
        I = o.I
        for _ in range(400):
            st, I = o.source(dt, I)
            assert st == 0
        T = o.temperature()
        assert abs(T.mean() / T_bal - 1) < 1e-9
        assert abs(T.mean() / g["T_eq_paper"] - 1) < 5e-3


def _ode_source_cell(prob, c, I0, dt, steps):
    """RK4 of the comoving source ODE of Eq. (com radiative source) and
    Eq. (com rad thermal) for one cell with the frame velocity frozen."""
    d, w = prob.dirs, prob.weights
    rho = prob.rho[c]
    v = prob.m[c] / rho
    # Sec. 2.3: Gamma = gamma (1 - v . n / c), gamma = 1 for the first-order problem
    gam = 1 / np.sqrt(1 - v @ v / prob.c ** 2) if prob.boost else 1.0
    G = gam * (1 - d @ v / prob.c)
    wc = w / G ** 2
    wc /= wc.sum()
    rcv = rho * prob.r_gas / (prob.gamma_gas - 1)
    kin = 0.5 * np.sum(prob.m[c] ** 2) / rho
    T = (prob.e[c] - kin) / rcv
    y = np.concatenate([G ** 4 * I0, [T]])
    kP0, kJ0, kS = prob.kappa_P[c], prob.kappa_J[c], prob.kappa_s[c]
    bP, bJ, Tr = getattr(prob, "beta_P", 0.0), getattr(prob, "beta_J", 0.0), getattr(prob, "T_ref", 1.0)

    def f(y):
        It, T = y[:-1], y[-1]
        # opacities at the current temperature (Sec. 2.3: temperature-dependent opacity)
        kP, kJ = kP0 * (T / Tr) ** bP, kJ0 * (T / Tr) ** bJ
        J = wc @ It
        dI = G * prob.cbar * rho * (kP * prob.a_rad * T ** 4 / (4 * np.pi) + kS * J - (kJ + kS) * It)
        dT = -prob.c * rho * (kP * prob.a_rad * T ** 4 - 4 * np.pi * kJ * J) / rcv
        return np.concatenate([dI, [dT]])

    h = dt / steps
    for _ in range(steps):
        k1 = f(y); k2 = f(y + h / 2 * k1); k3 = f(y + h / 2 * k2); k4 = f(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y[:-1] / G ** 4, y[-1]


def _heavy_gas(prob, H=1e6):
    """The same radiation problem (rho kappa, rho c_v, v and T unchanged) with
    the gas H times heavier, so that the radiation force leaves the frame
    velocity frozen, as the ODE reference assumes."""
    v = prob.m / prob.rho[:, None]
    T = (prob.e - 0.5 * np.sum(prob.m ** 2, 1) / prob.rho) * (prob.gamma_gas - 1) / (
        prob.rho * prob.r_gas)
    prob.rho = prob.rho * H
    prob.kappa_P, prob.kappa_J, prob.kappa_s = prob.kappa_P / H, prob.kappa_J / H, prob.kappa_s / H
    prob.r_gas = prob.r_gas / H
    prob.m = np.ascontiguousarray(prob.rho[:, None] * v)
    prob.e = prob.rho * prob.r_gas * T / (prob.gamma_gas - 1) + 0.5 * np.sum(prob.m ** 2, 1) / prob.rho
    return prob


@pytest.mark.parametrize("vscale,boost,opacity", [(0.0, 0, None), (0.05, 0, None), (0.25, 1, None),
                                                  (0.05, 0, (-3.0, 1.0, 1.0)),
                                                  (0.0, 0, (2.0, -1.0, 0.7))])
def test_implicit_source_converges_to_subcycled_explicit(vscale, boost, opacity):
    """8-cell mesh: N implicit source substeps approach a finely subcycled
    explicit (RK4) integration of the source ODE at first order in dt/N.  With
    the transformation to all orders (|v|/c up to 0.43, gamma up to 1.11) the
    gas is made heavy so that the frame velocity stays frozen; there the
    first-order update stalls at ~1e-2 against the all-orders ODE.  With
    temperature-dependent opacities the ODE takes both at the running
    temperature, the scheme kappa_P at T^{n+1} and kappa_J at T^n."""
    prob = randomise(make(n=(2, 2, 2), order=4, cbar=5.0, c=50.0), seed=4, v_scale=vscale,
                     kinds=False)
    if boost:
        prob = _heavy_gas(prob)
    prob.boost = boost
    if opacity is not None:
        # kappa_P ~ T^beta_P at T^{n+1} and kappa_J ~ T^beta_J at T^n in the scheme,
        # both at the running temperature in the ODE (cell temperatures 0.56 - 1.87)
        prob.beta_P, prob.beta_J, prob.T_ref = opacity
    I_start = prob.initial_intensity()
    dt = 0.02
    ref = [_ode_source_cell(prob, c, I_start[c], dt, 4000) for c in range(prob.n_cells)]
    errs = []
    for nsub in (8, 16, 32):
        o = oracle.Oracle(prob)
        I = I_start.copy()
        for _ in range(nsub):
            st, I = o.source(dt / nsub, I)
            assert st == 0
        err = max(np.abs(I[c] - ref[c][0]).max() / np.abs(ref[c][0]).max()
                  for c in range(prob.n_cells))
        errs.append(err)
    assert errs[-1] < 0.05
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


# ---------------------------------------------------------------- conservation (P3)
def test_energy_momentum_conserved_to_roundoff():
    """Sec. 2.3.1: E_gas + (c/cbar) E_r and rho v + F_r/(c cbar) are conserved,
    with the boundary / emitter tallies closing the budget; c != cbar,
    moving cells, scattering and a moving mesh all included."""
    prob = randomise(make(n=(4, 3, 5), order=6, cbar=10.0, c=100.0, w=(0.3, 0.1, 0.0)), seed=9)
    o = oracle.Oracle(prob)
    dt = 0.9 / o.positivity()
    t0 = o.totals()
    assert o.run(20, dt) == 0
    t1 = o.totals()
    assert abs(t1[12] - t0[12]) < 1e-13 * abs(t0[12])
    scale = np.abs(t0[3:12]).sum() + np.abs(t1[3:12]).sum()
    assert np.abs(t1[13:16] - t0[13:16]).max() < 1e-13 * scale
    assert abs(t1[0] - t0[0]) > 1e-6 * abs(t0[12])  # real exchange happened


def test_momentum_transfer_beamed_radiation():
    """Sec. 3.2: only rays with cos(theta) >= 0.8 to +x populated; the gas
    picks up +x momentum and total momentum is conserved (the paper shows
    4e-4; the discrete scheme conserves it to round-off)."""
    d, _ = level_symmetric(6)
    q0 = (d[:, 0] >= 0.8).astype(float) * 4.0
    prob = make(n=(4, 4, 4), order=6, cbar=100.0, c=100.0, kP=1.0, kJ=1.0, q0=q0,
                J0=1.0 / (4 * np.pi))
    o = oracle.Oracle(prob)
    dt = o.cfl_dt()
    t0 = o.totals()
    assert t0[6] > 0 and abs(t0[3]) == 0
    assert o.run(50, dt) == 0
    t1 = o.totals()
    assert t1[3] > 0.1 * t0[6]
    assert abs(t1[13] - t0[13]) < 1e-13 * t0[6]


def test_shadow_behind_opaque_sphere():
    """Sec. 3.5: a beam from the -y layer is stopped by an opaque sphere;
    cells in its geometric shadow stay dark while cells in the beam before
    the sphere are lit."""
    from paper_2002_08377_gb300.inputs import shadows
    prob = shadows(n=20, steps=60)
    N = prob.n_cells
    x = prob.mesh.points
    # one sphere in beam 1's path at y = 0.35, nothing else
    ctr = np.array([0.35 + 0.35 * np.tan(np.pi / 6), 0.35, 0.5])
    kap = np.full(N, 1e-3)
    kap[np.sum((x - ctr) ** 2, 1) < 0.12 ** 2] = 1e3
    prob.kappa_P, prob.kappa_J = kap, kap.copy()
    prob.kind[prob.kind == 2] = 0
    prob.emit_rate[:] = 0
    prob.I0[2] = 0.0
    o = oracle.Oracle(prob)
    dt = o.cfl_dt()
    assert o.run(60, dt) == 0
    E, _, _ = o.moments()
    b = np.array([0.5, np.sqrt(3) / 2, 0.0])
    rel = x - np.array([0.35, 0.0, 0.5])
    along = rel @ b
    perp = np.linalg.norm(rel - along[:, None] * b, axis=1)
    beam = (perp < 0.03) & (np.abs(x[:, 2] - 0.5) < 0.1)
    lit = beam & (along > 0.1) & (along < 0.2)
    dark = beam & (along > 0.6) & (along < 0.8)
    assert lit.any() and dark.any()
    # first-order upwinding on a 20^3 mesh diffuses the beam edge into the
    # umbra; the shadow is still darker than the beam by a factor > 50
    assert E[dark].max() < 2e-2 * E[lit].mean()
    assert E[dark].max() > 0.0


# ---------------------------------------------------------------- diffusion limit
def _diffusion_gaussian_error(N, v, chi=125.0, dx=0.08, rho0=1e6, integrator=0):
    """Sec. 3.3 setup, first-order scheme: a quasi-1-D periodic box (N x 3 x 3
    cubic cells, lattice jitter 1e-6 of the spacing), one angle per octant,
    a scattering medium of total opacity rho kappa_s = chi, c = cbar, the gas
    heavy enough (rho = 1e6) that radiation neither accelerates nor heats it
    (the paper does not evolve the hydrodynamics), flow and mesh at v = w.
    The radiation starts isotropic in the comoving frame with
    E_r = exp(-x^2/dx^2) + exp(-10) (the paper's floor) and runs until the
    diffusion solution of Eq. (diff analytic), D = cbar / (3 chi), has
    doubled its variance.  Returns the L1 error of E_r relative to the
    Gaussian's own L1 norm, in the mesh frame (cells move with w = v)."""
    from paper_2002_08377_gb300.inputs import Problem
    h = 1.0 / N
    mesh = build_mesh((N, 3, 3), box=(1.0, 3 * h, 3 * h), jitter=1e-6, seed=5)
    mesh.face_w = np.ascontiguousarray(np.tile([v, 0.0, 0.0], (mesh.n_faces, 1)))
    dirs, wt = level_symmetric(2)
    n, A = mesh.n_cells, dirs.shape[0]
    x = mesh.cell_centroid[:, 0] - 0.5
    E0 = np.exp(-x ** 2 / dx ** 2) + np.exp(-10.0)
    rho = np.full(n, rho0)
    vel = np.zeros((n, 3))
    vel[:, 0] = v
    m = rho[:, None] * vel
    e = rho * 1.5 + 0.5 * rho * v * v  # T = 1, gamma = 5/3
    z = np.zeros(n)
    gamma = 1.0 - dirs[:, 0] * v  # c = 1
    prob = Problem("diffusion-gaussian", mesh, dirs, wt, 1.0, 1.0, 1.0, 5.0 / 3.0, 1.0, 0.3, 0,
                   rho, e, m, z.copy(), z.copy(), np.full(n, chi / rho0), np.zeros(n, np.uint8),
                   z.copy(), z.copy(), z.copy(), np.full(n, -1, np.int32), np.zeros((1, A)),
                   E0 / (4 * np.pi), 1.0 / gamma ** 4, integrator=integrator)
    o = oracle.Oracle(prob)
    D = 1.0 / (3.0 * chi)
    t_end = dx ** 2 / (4.0 * D)
    steps = int(np.ceil(t_end / o.cfl_dt()))
    assert o.run(steps, t_end / steps) == 0
    E = o.moments()[0]
    s = 1.0 + 4.0 * D * t_end / dx ** 2
    Ea = np.exp(-x ** 2 / (dx ** 2 * s)) / np.sqrt(s) + np.exp(-10.0)
    return np.sum(np.abs(E - Ea)) / np.sum(Ea - np.exp(-10.0))


@pytest.mark.parametrize("v", [0.0, 0.1])
def test_diffusion_gaussian_converges_at_first_order(v):
    """Sec. 3.3 (dynamic diffusion) with Eq. (diff analytic): in an optically
    thick scattering medium (cell optical depth 1 to 0.25) the piecewise-
    constant upwind step plus the implicit source converges to the diffusion
    solution at first order in the cell size, static or moving with the
    flow (Sec. 3.6 states first-order convergence of the method)."""
    errs = [_diffusion_gaussian_error(N, v) for N in (128, 256, 512)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[0] > errs[1] > errs[2], errs
    assert np.all((orders > 0.75) & (orders < 1.3)), (errs, orders)
    assert errs[2] < 0.06, errs


# ---------------------------------------------------------------- linear modes
def _linear_system(dirs, wt, k, cbar, c, chi, rcv, a=1.0, T=1.0):
    """The radiation-thermal equations linearised about rest and equilibrium
    (I = aT^4/4pi isotropic, v = 0) for a perturbation exp(ikx), continuous in
    space and time: per angle
      d dI_a/dt = -i k cbar n_ax dI_a + cbar chi (4aT^3/4pi dT - dI_a),
    and for the gas (rho c_v) d dT/dt = c chi (4pi dJ - 4aT^3 dT), dJ = sum w dI
    (Eqs. time evolution, com radiative source, tgas with kappa_P = kappa_J,
    kappa_s = 0).  Returns the (A+1) x (A+1) matrix."""
    A = len(wt)
    M = np.zeros((A + 1, A + 1), complex)
    M[np.arange(A), np.arange(A)] = -1j * k * cbar * dirs[:, 0] - cbar * chi
    M[:A, A] = cbar * chi * 4 * a * T ** 3 / (4 * np.pi)
    M[A, :A] = (c / rcv) * 4 * np.pi * chi * wt
    M[A, A] = -(c / rcv) * chi * 4 * a * T ** 3
    return M


def _measured_mode(N, chi, cbar=1.0, c=100.0, amp=1e-6):
    """Sec. 3.6 setup with the hydrodynamics frozen: a quasi-1-D periodic box
    (N x 3 x 3 cells, lattice jitter 10 % of the spacing), one angle per
    octant, k = 2 pi / L_x, cbar = c / 100, P_rad of the order of P_gas.  The
    gas is made inertially heavy (rho = 1e8) with its heat capacity kept
    (rho c_v = 1.5 through r_gas = 1e-8) and rho kappa = chi, so radiation
    cannot move it (the paper fixes the flow for the radiation part).  The
    slowest-decaying eigenvector of the linear system with an E_r component
    is laid on the mesh at amplitude 1e-6; the oracle's E_r Fourier
    coefficient at k gives the measured rate lambda = log(c2/c1)/(t2 - t1)."""
    from paper_2002_08377_gb300.inputs import Problem
    h = 1.0 / N
    mesh = build_mesh((N, 3, 3), box=(1.0, 3 * h, 3 * h), jitter=0.1, seed=5)
    dirs, wt = level_symmetric(2)
    n, A = mesh.n_cells, dirs.shape[0]
    rho0, r_gas = 1e8, 1e-8
    rcv = rho0 * r_gas / (2.0 / 3.0)
    k = 2 * np.pi
    lam, vec = np.linalg.eig(_linear_system(dirs, wt, k, cbar, c, chi, rcv))
    with_E = np.abs(vec[:A].T @ wt) > 1e-3 * np.abs(vec[:A].T @ wt).max()
    j = np.flatnonzero(with_E)[np.argmax(lam[with_E].real)]
    v = vec[:, j] / (4 * np.pi * (vec[:A, j] @ wt))  # unit E_r amplitude
    x = mesh.cell_centroid[:, 0]
    ph = np.exp(1j * k * x)
    I = 1 / (4 * np.pi) + amp * np.real(np.outer(ph, v[:A]))
    T = 1.0 + amp * np.real(ph * v[A])
    z = np.zeros(n)
    rho = np.full(n, rho0)
    prob = Problem("linear-mode", mesh, dirs, wt, cbar, c, 1.0, 5.0 / 3.0, r_gas, 0.3, 0, rho,
                   rho * r_gas * T / (2.0 / 3.0), np.zeros((n, 3)), np.full(n, chi / rho0),
                   np.full(n, chi / rho0), z.copy(), np.zeros(n, np.uint8), z.copy(), z.copy(),
                   z.copy(), np.full(n, -1, np.int32), np.zeros((1, A)), np.full(n, 1 / (4 * np.pi)),
                   np.ones(A))
    prob.initial_intensity = lambda dtype=np.float64, _I=I: np.ascontiguousarray(_I.astype(dtype))
    o = oracle.Oracle(prob)
    V = mesh.cell_volume

    def coefficient():
        return np.sum(V * (o.moments()[0] - 1.0) * np.conj(ph)) / np.sum(V)

    t_end = min(1.0, 2.0 / abs(lam[j].real))
    steps = int(np.ceil(t_end / o.cfl_dt()))
    dt = t_end / steps
    n1 = steps // 4  # let the other (fast) discrete modes die out first
    assert o.run(n1, dt) == 0
    c1 = coefficient()
    assert o.run(steps - n1, dt) == 0
    return lam[j], np.log(coefficient() / c1) / ((steps - n1) * dt)


@pytest.mark.parametrize("chi", [1.0, 10.0])
def test_linear_radiation_thermal_mode_converges_at_first_order(chi):
    """Sec. 3.6 (linear wave, reading: radiation-thermal part with the flow
    frozen): the decay rate and phase speed of the slowest E_r mode converge
    to the eigenvalue of the linearised equations at first order in the cell
    size -- a propagating, damped mode at optical depth 1 per wavelength
    (chi = 1) and a diffusive one at optical depth 10."""
    errs = []
    for N in (32, 64, 128):
        lam, measured = _measured_mode(N, chi)
        errs.append(abs(measured - lam) / abs(lam))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 0.8) & (orders < 1.25)), (errs, orders)
    assert errs[-1] < 0.08, errs
