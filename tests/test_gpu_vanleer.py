"""GPU parity of the van Leer step with limited linear reconstruction
(integrator RT_VAN_LEER) against the oracle's van Leer step, through the C
ABI, with the tolerances of the first-order path: RT_FP64 per intensity to
a relative 1e-12, RT_FP32 in L1 of E_r to 1e-5 with total energy conserved
to 1e-6."""
import numpy as np
import pytest

import oracle
from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from paper_2002_08377_gb300.inputs import diffusion, shadows
from tests._problems import make, randomise

pytestmark = pytest.mark.gpu

FP64_REL = 1e-12
FP32_L1 = 1e-5
FP32_ENERGY = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()
    capi.load()


def _solver(prob, precision):
    from paper_2002_08377_gb300.solver import RTSolver
    return RTSolver.from_problem(prob, precision)


def _rel(g, o):
    g = np.asarray(g, np.float64)
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-300)))


def _l1(g, o):
    return float(np.sum(np.abs(g - o)) / np.sum(np.abs(o)))


def _run(prob, precision, steps, dt_frac=0.5):
    prob.integrator = capi.RT_VAN_LEER
    o = oracle.Oracle(prob)
    dt = dt_frac / o.positivity()
    g = _solver(prob, precision)
    t0 = g.totals()
    assert o.run(steps, dt) == oracle.ORC_OK
    g.run(steps, dt)
    return o, g, t0


def _check(o, g, precision, t0=None):
    if precision == "fp64":
        assert _rel(g.get_intensity(), o.I) < FP64_REL
        e, m, _ = g.gas()
        assert _rel(e, o.e) < FP64_REL
        E, _, _ = o.moments()
        scale = np.abs(o.m).max() + E.max() / o.prob.cbar
        assert np.abs(m - o.m).max() < FP64_REL * scale
    else:
        assert _l1(g.moments()[0], o.moments()[0]) < FP32_L1
        assert _l1(g.gas()[0], o.e) < FP32_L1
        t1 = g.totals()
        assert abs(t1[12] - t0[12]) < FP32_ENERGY * abs(t0[12])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("moving", [False, True])
def test_van_leer_random_problem(precision, moving):
    """Random opacities, anisotropic intensities, moving gas, boundary and
    emitter cells, scattering; static or moving mesh; S6 and S8."""
    w = (0.2, -0.1, 0.15) if moving else None
    for order, n in ((6, (9, 7, 5)), (8, (6, 5, 7))):
        prob = randomise(make(n=n, order=order, cbar=10.0, c=100.0, w=w), seed=5 + order)
        o, g, t0 = _run(prob, precision, 20)
        _check(o, g, precision, t0)
        g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_van_leer_diffusion_shape(precision):
    """Diffusion workload at 20^3 (moving mesh and gas, stiff cells)."""
    o, g, t0 = _run(diffusion(n=20, steps=40), precision, 40)
    _check(o, g, precision, t0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_van_leer_shadows_full_size_one_step(precision):
    """Shadows workload at full size (128^3 cells, 80 angles): one van Leer
    step, every cell compared."""
    prob = shadows()
    prob.integrator = capi.RT_VAN_LEER
    o = oracle.Oracle(prob)
    dt = o.cfl_dt()
    g = _solver(prob, precision)
    t0 = g.totals()
    assert o.step(dt) == oracle.ORC_OK
    g.step(dt)
    _check(o, g, precision, t0)
    g.close()


def test_van_leer_state_rejects_the_adjoint():
    """The hand-written adjoint reverses the first-order step only."""
    import torch
    prob = make(n=(4, 4, 4), order=4)
    prob.integrator = capi.RT_VAN_LEER
    g = _solver(prob, "fp64")
    N, A = prob.n_cells, prob.n_angles
    t = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.RTError) as err:
        g.adjoint_step(0.01, t(N, A), t(N), t(N, 3), t(N, A), t(N), t(N, 3), t(N), t(N))
    assert err.value.code == capi.RT_ERR_STATE


def _custom_angles(prob, n_pairs, seed):
    """The problem on n_pairs random antipodal pairs of directions with equal
    weights (angle counts the level-symmetric sets do not reach: 32 rows take
    one quad per thread and no tail, 112 three quads and a tail)."""
    rng = np.random.default_rng(seed)
    up = rng.normal(size=(n_pairs, 3))
    up /= np.linalg.norm(up, axis=1, keepdims=True)
    prob.dirs = np.ascontiguousarray(np.concatenate([up, -up]))
    A = 2 * n_pairs
    prob.weights = np.full(A, 1.0 / A)
    prob.q0 = np.ones(A)
    prob.I0 = np.zeros((1, A))
    return prob


@pytest.mark.parametrize("n_pairs", [16, 56], ids=["A32", "A112"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vanleer_custom_angle_sets(n_pairs, precision):
    base = make(n=(7, 6, 5), order=2, cbar=10.0, c=100.0, w=(0.3, -0.1, 0.2))
    prob = randomise(_custom_angles(base, n_pairs, 3), seed=6)
    o, g, t0 = _run(prob, precision, 10)
    _check(o, g, precision, t0)

