"""GPU parity of moving meshes (Sec. 2.2) through the C ABI against the FP64
oracle: per-face velocities from the generators' velocities (the
face-velocity equation), and the geometric conservation law (rt_params.gcl
= 1) that lets the cell volumes follow them.  RT_FP64 per intensity to a
relative 1e-12 (totals, which use the evolved volumes, too); RT_FP32 in L1
of E_r to 1e-5."""
import numpy as np
import pytest

import oracle
from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from tests._problems import make, randomise
from tests.test_gpu_parity import FP32_L1, check_fp32, check_fp64, l1_rel, solver
from tests.test_oracle_moving_mesh import _moving

pytestmark = pytest.mark.gpu

FP32_ENERGY = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()
    capi.load()


# ---------------------------------------------------------------- per-face velocities
def _rotating(n, order, seed):
    """A mesh in rigid rotation about the box centre: face velocities from
    the generators' velocities by the face-velocity equation (every face has
    its own w; the field jumps across the periodic boundary, which the
    transport takes like any other face velocity)."""
    prob = randomise(make(n=n, order=order, cbar=10.0, c=100.0), seed=seed)
    m = prob.mesh
    Om = np.array([0.4, -0.7, 0.9])
    m.face_w = m.face_velocity(np.cross(Om, m.points - 0.5 * m.box))
    return prob


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rotating_mesh(precision):
    prob = _rotating((9, 7, 5), 8, 3)
    o = oracle.Oracle(prob)
    g = solver(prob, precision)
    t0 = g.totals()
    dt = o.cfl_dt()
    assert o.run(30, dt) == oracle.ORC_OK
    g.run(30, dt)
    if precision == "fp64":
        check_fp64(o, g)
    else:
        check_fp32(o, g)
        t1 = g.totals()
        assert abs(t1[12] - t0[12]) < FP32_ENERGY * abs(t0[12])



# ---------------------------------------------------------------- geometric conservation law
def _gcl_problem(order=8, seed=3):
    """Opacities, scattering, boundary and emitter cells, moving gas, and a
    mesh expanding and rotating with per-face velocities."""
    prob = randomise(_moving(n=(9, 7, 5), order=order, seed=seed), seed=seed)
    return prob


@pytest.mark.parametrize("order", [6, 8])
def test_gcl_fp64(order):
    prob = _gcl_problem(order)
    o = oracle.Oracle(prob)
    g = solver(prob, "fp64")
    dt = 0.5 / o.positivity()
    assert o.run(30, dt) == oracle.ORC_OK
    g.run(30, dt)
    check_fp64(o, g)
    t_o, t_g = o.totals(), g.totals()
    assert np.abs(t_g - t_o).max() < 1e-12 * np.abs(t_o).max()
    assert np.abs(o.vol - prob.mesh.cell_volume).max() > 1e-3 * prob.mesh.cell_volume.max()


def test_gcl_fp32():
    prob = _gcl_problem(8, 4)
    o = oracle.Oracle(prob)
    g = solver(prob, "fp32")
    dt = 0.5 / o.positivity()
    assert o.run(30, dt) == oracle.ORC_OK
    g.run(30, dt)
    check_fp32(o, g)
    t_o, t_g = o.totals(), g.totals()
    assert abs(t_g[12] - t_o[12]) < FP32_ENERGY * abs(t_o[12])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-5)])
def test_gcl_preserves_a_uniform_field(precision, tol):
    prob = _moving()
    prob.q0 = np.random.default_rng(2).uniform(0.5, 2.0, prob.n_angles)
    g = solver(prob, precision)
    I0 = g.get_intensity().astype(np.float64)
    dt = 0.5 / oracle.Oracle(prob).positivity()
    g.run(5, dt)
    I = g.get_intensity().astype(np.float64)
    assert np.abs(I - I0).max() < tol * I0.max()


def test_gcl_state_round_trip_keeps_the_volumes():
    prob = _gcl_problem(6, 5)
    g = solver(prob, "fp64")
    dt = 0.5 / oracle.Oracle(prob).positivity()
    g.run(5, dt)
    buf = g.get_state()
    t5 = g.totals()
    g.run(5, dt)
    t10 = g.totals()
    g.set_state(buf)
    assert np.abs(g.totals() - t5).max() <= 1e-15 * np.abs(t5).max()
    g.run(5, dt)
    assert np.abs(g.totals() - t10).max() <= 1e-15 * np.abs(t10).max()


def _kv(prob):
    """max_a sum_f max(u_fa, 0) per cell (outward normals), numpy."""
    m = prob.mesh
    kv = np.zeros(m.n_cells)
    d = prob.dirs
    for c in range(m.n_cells):
        acc = np.zeros(prob.n_angles)
        for k in range(m.cell_face_ptr[c], m.cell_face_ptr[c + 1]):
            e = m.cell_face_idx[k]
            f, sg = (e, 1.0) if e >= 0 else (-e - 1, -1.0)
            n = sg * m.face_normal[f]
            u = prob.cbar * m.face_area[f] * (d @ n) - m.face_area[f] * (m.face_w[f] @ n)
            acc += np.maximum(u, 0.0)
        kv[c] = acc.max()
    return kv


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gcl_reports_a_shrinking_cell_past_its_positivity_limit(precision):
    """A contracting mesh at dt = 0.9 of the creation limit: the step in
    which some cell's volume has shrunk below dt max_a sum_f u+ is reported
    as RT_ERR_CFL (the steps before it are not)."""
    prob = _moving(n=(6, 5, 7), lam=-2.0, om=(0.0, 0.0, 0.0))
    o = oracle.Oracle(prob)
    dt = 0.9 / o.positivity()
    kv = _kv(prob)
    first = None
    for n in range(200):
        if np.any(o.vol < dt * kv * (1 - 1e-4)):
            first = n
            break
        assert o.step(dt) == oracle.ORC_OK
    assert first is not None and first >= 3
    g = solver(prob, precision)
    g.run(first - 1, dt)
    with pytest.raises(capi.RTError) as err:
        g.run(2, dt)
    assert err.value.code == capi.RT_ERR_CFL
