"""GPU cases that reach what the jittered workloads do not:

* a cube lattice, where the transport must be exactly the textbook
  donor-cell (first-order upwind) scheme, with directions along the lattice
  axes so that u = 0 on every face parallel to them (the upwind tie of
  Sec. 2.2 carries no flux);
* the worked example of Sec. 3.1 in CGS units (a parsec box of atomic
  hydrogen at rho = 1e-15 g/cc, gas at 10 K, radiation at 200 K, cbar = c):
  the FP64 step and its adjoint at physical scale, against the oracle, the
  equilibrium temperature of the energy balance, and the clean refusal of
  an FP32 state whose face coefficients cbar A overflow float.
"""
import dataclasses
import os

import numpy as np
import pytest

import oracle
from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from tests._problems import make

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()
    capi.load()


def solver(prob, precision, **kw):
    from paper_2002_08377_gb300.solver import RTSolver
    return RTSolver.from_problem(prob, precision, **kw)


def axis_diagonal_set():
    """14 directions: the 6 lattice axes and the 8 cube diagonals, ordered
    so that direction a + 7 is -(direction a); weights 1/12 (axes) and
    1/16 (diagonals), which sum to one."""
    s = 1.0 / np.sqrt(3.0)
    half = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (s, s, s), (s, s, -s), (s, -s, s), (-s, s, s)]
    d = np.array(half + [tuple(-x for x in v) for v in half], np.float64)
    w = np.array([1 / 12] * 3 + [1 / 16] * 4, np.float64)
    return d, np.concatenate([w, w])


def donor_cell(I, n, dirs, nu):
    """Textbook donor-cell update of a periodic n[0] x n[1] x n[2] lattice
    (cell (i, j, k) at row i + n0 (j + n1 k)), Courant numbers nu per axis
    direction: I - nu sum_d (n_d^+ (I - I_{-e_d}) + n_d^- (I_{+e_d} - I))."""
    n0, n1, n2 = n
    A = I.shape[1]
    F = I.reshape(n2, n1, n0, A)  # [k][j][i][a]
    out = F.copy()
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        up = np.maximum(dirs[:, d], 0.0)
        dn = np.minimum(dirs[:, d], 0.0)
        minus = np.roll(F, 1, axis=ax)   # neighbour at -e_d
        plus = np.roll(F, -1, axis=ax)   # neighbour at +e_d
        out = out - nu[d] * (up * (F - minus) + dn * (plus - F))
    return out.reshape(-1, A)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_cube_lattice_is_donor_cell_with_ties(precision, tol):
    """One step with no matter coupling (kappa = 0, v = 0: the source step
    is the identity) on an unjittered 6 x 5 x 4 lattice of unequal spacings
    is the donor-cell scheme; axis directions meet faces parallel to them
    with u = 0 exactly."""
    n = (6, 5, 4)
    prob = make(n=n, jitter=0.0, cbar=10.0, c=10.0, kP=0.0, kJ=0.0, kS=0.0)
    dirs, w = axis_diagonal_set()
    rng = np.random.default_rng(4)
    I = rng.uniform(0.1, 2.0, (prob.n_cells, len(w)))
    prob = dataclasses.replace(prob, dirs=dirs, weights=w, q0=np.ones(len(w)),
                               I0=np.zeros((1, len(w))))
    prob.initial_intensity = lambda dtype=np.float64, _I=I: np.ascontiguousarray(_I.astype(dtype))
    h = 1.0 / np.array(n, float)  # unit box: spacing per axis
    g = solver(prob, precision)
    dt = 0.9 * g.dt_limits()[1]
    g.step(dt)
    out = g.get_intensity().astype(np.float64)
    g.close()
    # the mesh builder's cells in the row order of donor_cell
    ix, iy, iz = prob.mesh.lattice_index()
    order = np.argsort(ix + n[0] * (iy + n[1] * iz))
    want = donor_cell(I[order], n, dirs, prob.cbar * dt / h)
    got = out[order]
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


# ------------------------------------------------------------------ CGS, Sec. 3.1
def _golden():
    vals = {}
    with open(os.path.join(GOLDEN, "thermal_equilibrium_cgs.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


PC = 3.0856775814913673e18  # cm
KB, MP, A_RAD, C = 1.380649e-16, 1.67262192e-24, 7.565733e-15, 2.99792458e10


def scaled_mesh(mesh, L):
    """The same tessellation with every length multiplied by L."""
    return dataclasses.replace(
        mesh, box=mesh.box * L, points=mesh.points * L, cell_volume=mesh.cell_volume * L ** 3,
        cell_centroid=mesh.cell_centroid * L, face_area=mesh.face_area * L ** 2,
        face_centroid=mesh.face_centroid * L)


def cgs_problem(kappa, n=6):
    g = _golden()
    prob = make(n=(n, n, n), order=6, cbar=C, c=C, a_rad=A_RAD, r_gas=KB / MP, rho=g["rho"],
                T=g["T_gas"], kP=kappa, kJ=kappa, J0=A_RAD * g["T_rad"] ** 4 / (4 * np.pi))
    return dataclasses.replace(prob, mesh=scaled_mesh(prob.mesh, PC)), g


@pytest.mark.parametrize("kappa", [1.0, 100.0])
def test_cgs_worked_example_fp64(kappa):
    """The FP64 state at physical scale (cbar A ~ 1e45, dt/V ~ 1e-48) follows
    the oracle per intensity to 1e-12 over 30 Courant steps, and both reach
    the equilibrium temperature of the energy balance (101.33 K with these
    constants; the paper prints 101.7 K)."""
    from scipy.optimize import brentq
    prob, gold = cgs_problem(kappa)
    o = oracle.Oracle(prob)
    dt = o.cfl_dt()
    g = solver(prob, "fp64")
    assert o.run(30, dt) == 0
    g.run(30, dt)
    I = g.get_intensity()
    assert np.max(np.abs(I - o.I) / np.abs(o.I)) < 1e-12
    e, m, _ = g.gas()
    assert np.max(np.abs(e - o.e) / np.abs(o.e)) < 1e-12
    rcv = gold["rho"] * KB / (MP * (5.0 / 3.0 - 1.0))
    E0 = rcv * gold["T_gas"] + A_RAD * gold["T_rad"] ** 4
    T_bal = brentq(lambda T: rcv * T + A_RAD * T ** 4 - E0, 1.0, 1e3)
    kin = 0.5 * np.sum(m ** 2, 1) / prob.rho
    T = (e - kin) * (2.0 / 3.0) / (prob.rho * prob.r_gas)
    assert np.abs(T / T_bal - 1).max() < 1e-6
    g.close()


def test_cgs_worked_example_adjoint_fp64():
    """One reverse step of the FP64 state at physical scale against the
    oracle's discrete adjoint (1e-10)."""
    import torch
    prob, _ = cgs_problem(1.0, n=5)
    rng = np.random.default_rng(3)
    prob.initial_intensity = (lambda dtype=np.float64, _I=prob.initial_intensity() *
                              rng.uniform(0.5, 1.5, (prob.n_cells, prob.n_angles)):
                              np.ascontiguousarray(_I.astype(dtype)))
    o = oracle.Oracle(prob)
    dt = o.cfl_dt()
    N, A = prob.n_cells, prob.n_angles
    lI1, le1, lm1 = rng.standard_normal((N, A)), rng.standard_normal(N), rng.standard_normal((N, 3))
    gP_o, gJ_o = np.zeros(N), np.zeros(N)
    lI_o, le_o, _ = o.adjoint_step(dt, o.I, o.e, o.m, lI1, le1, lm1, gP_o, gJ_o)
    g = solver(prob, "fp64")
    dev = lambda x: torch.tensor(x, device="cuda")
    gP = torch.zeros(N, dtype=torch.float64, device="cuda")
    gJ = torch.zeros_like(gP)
    lI, le, _ = g.adjoint_step(dt, dev(o.I), dev(o.e), dev(o.m), dev(lI1), dev(le1), dev(lm1), gP, gJ)
    for x, y in ((lI, lI_o), (le, le_o), (gP, gP_o), (gJ, gJ_o)):
        x = x.cpu().numpy()
        assert np.abs(x - y).max() <= 1e-10 * np.abs(y).max()
    g.close()


def test_cgs_fp32_refused_cleanly():
    """An FP32 state of the parsec box would overflow float in cbar A; the
    library refuses it at creation with RT_ERR_ARG instead of stepping to a
    non-finite state."""
    prob, _ = cgs_problem(1.0, n=4)
    with pytest.raises(capi.RTError) as ei:
        solver(prob, "fp32")
    assert ei.value.code == capi.RT_ERR_ARG
