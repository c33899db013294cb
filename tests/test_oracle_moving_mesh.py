"""CPU pins of the oracle's moving mesh (Sec. 2.2): face velocities from the
velocities of the mesh-generating points, and the geometric conservation
law (GCL) that changes the cells' volumes with the face velocities.

With the GCL (problem flag `gcl`) each step takes V^{n+1} = V^n + dt sum_f
A_f w_f . n_f and the conservative moving-cell transport V^{n+1} I* = V^n I
- dt sum_f u I_up.  The pins: a uniform field stays uniform on any moving
mesh (free-stream preservation; without the GCL it drifts), sum_c V_c I_ca is
conserved for every angle, and the interior cells of a uniformly expanding
(and rotating) mesh grow exactly by 1 + 3 lambda dt per step (the divergence
theorem on planar faces).
"""
import numpy as np
import pytest

import oracle
from paper_2002_08377_gb300.inputs import build_mesh
from tests._problems import make, randomise


def test_face_velocity_of_rigid_motion_and_expansion():
    """For generators moving with w(r) = b + Omega x r + lambda r (a rigid
    motion plus uniform expansion) the tessellation moves with the same
    field, so the normal velocity of every face at its centroid is
    w(x_f) . n_f; the face-velocity formula gives exactly that (faces that do
    not cross the periodic boundary, where the field is continuous).  A
    uniform field gives w_f = w on every face."""
    m = build_mesh((6, 5, 7), jitter=0.25, seed=5)
    rng = np.random.default_rng(8)
    b, Om, lam = rng.standard_normal(3), rng.standard_normal(3), 0.37

    def field(r):
        return b + np.cross(Om, r) + lam * r

    wf = m.face_velocity(field(m.points))
    inner = ~np.any(m.face_shift != 0, axis=1)
    assert inner.sum() > 100
    lhs = np.sum(wf * m.face_normal, axis=1)[inner]
    rhs = np.sum(field(m.face_centroid) * m.face_normal, axis=1)[inner]
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()
    # the correction term matters: the mean of the generators alone is off
    mean = 0.5 * (field(m.points[m.face_cells[:, 0]]) + field(m.points[m.face_cells[:, 1]]))
    off = np.abs(np.sum(mean * m.face_normal, axis=1)[inner] - rhs).max()
    assert off > 1e-3 * np.abs(rhs).max()
    wu = m.face_velocity(np.broadcast_to(b, (m.n_cells, 3)))
    assert np.abs(wu - b).max() < 1e-14 * np.abs(b).max()


def _moving(n=(6, 5, 7), lam=0.15, om=(0.4, -0.7, 0.9), gcl=1, seed=5, order=6, **kw):
    """No opacity (transport only), face velocities from generators moving
    with lam (r - r0) + Omega x (r - r0) (the field jumps across the periodic
    boundary, which the GCL takes like any other face velocity)."""
    prob = make(n=n, order=order, cbar=10.0, c=100.0, kP=0.0, kJ=0.0, kS=0.0, seed=seed, **kw)
    m = prob.mesh
    r = m.points - 0.5 * m.box
    m.face_w = m.face_velocity(lam * r + np.cross(np.asarray(om, float), r))
    prob.gcl = gcl
    return prob


@pytest.mark.parametrize("gcl", [1, 0])
def test_uniform_field_is_preserved_only_with_the_gcl(gcl):
    prob = _moving(gcl=gcl)
    rng = np.random.default_rng(2)
    prob.q0 = rng.uniform(0.5, 2.0, prob.n_angles)  # anisotropic, the same in every cell
    o = oracle.Oracle(prob)
    I0 = o.I.copy()
    dt = 0.5 / o.positivity()
    assert o.run(5, dt) == oracle.ORC_OK
    dev = np.abs(o.I - I0).max() / I0.max()
    if gcl:
        assert dev < 1e-13
    else:
        assert dev > 1e-3


def test_gcl_conserves_volume_integral_per_angle():
    prob = randomise(_moving(), seed=4, v_scale=0.0)
    prob.kappa_P[:] = prob.kappa_J[:] = prob.kappa_s[:] = 0.0
    prob.kind[:] = 0
    o = oracle.Oracle(prob)
    dt = 0.5 / o.positivity()
    s0 = o.vol @ o.I
    assert o.run(5, dt) == oracle.ORC_OK
    s1 = o.vol @ o.I
    assert np.abs(s1 - s0).max() < 1e-13 * np.abs(s0).max()
    assert np.abs(o.vol - prob.mesh.cell_volume).max() > 1e-3 * prob.mesh.cell_volume.max()


def test_gcl_volumes_follow_the_expansion():
    lam = 0.15
    prob = _moving(lam=lam)
    m = prob.mesh
    o = oracle.Oracle(prob)
    dt = 0.5 / o.positivity()
    assert o.step(dt) == oracle.ORC_OK
    per = np.any(m.face_shift != 0, axis=1)
    touched = np.zeros(m.n_cells, bool)
    touched[m.face_cells[per, 0]] = touched[m.face_cells[per, 1]] = True
    inner = ~touched
    assert inner.sum() > 20
    ratio = o.vol[inner] / m.cell_volume[inner]
    assert np.abs(ratio - (1 + 3 * lam * dt)).max() < 1e-12


def test_van_leer_and_adjoint_refuse_the_gcl():
    prob = _moving(n=(3, 3, 3), order=4)
    prob.integrator = 1
    with pytest.raises(ValueError):
        oracle.Oracle(prob).step(0.01)
    prob = _moving(n=(3, 3, 3), order=4)
    o = oracle.Oracle(prob)
    N, A = prob.n_cells, prob.n_angles
    z = np.zeros(N)
    with pytest.raises(ValueError):
        o.adjoint_step(0.01, o.I, o.e, o.m, np.ones((N, A)), z, np.zeros((N, 3)), z.copy(), z.copy())
