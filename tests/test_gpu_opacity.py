"""GPU parity of temperature-dependent opacities (rt_params beta_P, beta_J,
T_ref; Sec. 2.3's Newton-Raphson temperature solve) through the C ABI against
the FP64 oracle: RT_FP64 per intensity to a relative 1e-12, RT_FP32 in L1 of
E_r to 1e-5 with total energy conserved to 1e-6."""
import numpy as np
import pytest

import oracle
from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from tests._problems import make, randomise
from tests.test_gpu_parity import check_fp32, check_fp64, solver

pytestmark = pytest.mark.gpu

FP32_ENERGY = 1e-6
CASES = [(-3.0, 1.0, 1.0), (2.0, -1.0, 0.7)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()
    capi.load()


def _problem(betas, order=8, seed=5, w=(0.3, -0.1, 0.2)):
    prob = randomise(make(n=(9, 7, 5), order=order, cbar=10.0, c=100.0, w=w), seed=seed)
    prob.beta_P, prob.beta_J, prob.T_ref = betas
    return prob


@pytest.mark.parametrize("betas", CASES)
@pytest.mark.parametrize("order", [6, 8])
def test_fp64_temperature_dependent_opacity(betas, order):
    prob = _problem(betas, order)
    o = oracle.Oracle(prob)
    g = solver(prob, "fp64")
    dt = o.cfl_dt()
    assert o.run(30, dt) == oracle.ORC_OK
    g.run(30, dt)
    check_fp64(o, g)


@pytest.mark.parametrize("betas", CASES)
def test_fp32_temperature_dependent_opacity(betas):
    prob = _problem(betas, 8, 6)
    o = oracle.Oracle(prob)
    g = solver(prob, "fp32")
    t0 = g.totals()
    dt = o.cfl_dt()
    assert o.run(30, dt) == oracle.ORC_OK
    g.run(30, dt)
    check_fp32(o, g)
    t1 = g.totals()
    assert abs(t1[12] - t0[12]) < FP32_ENERGY * abs(t0[12])


def test_van_leer_temperature_dependent_opacity_fp64():
    prob = randomise(make(n=(6, 5, 7), order=6, cbar=10.0, c=100.0, w=(0.2, -0.1, 0.15)), seed=7)
    prob.beta_P, prob.beta_J, prob.T_ref = -3.0, 1.0, 1.0
    prob.integrator = capi.RT_VAN_LEER
    o = oracle.Oracle(prob)
    g = solver(prob, "fp64")
    dt = 0.5 / o.positivity()
    assert o.run(20, dt) == oracle.ORC_OK
    g.run(20, dt)
    check_fp64(o, g)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_equilibrium_with_equal_exponents(precision, tol):
    prob = make(n=(3, 4, 3), order=6, cbar=5.0, c=20.0, T=1.3, kP=2.0, kJ=2.0, kS=0.4)
    prob.beta_P, prob.beta_J, prob.T_ref = 1.5, 1.5, 0.6
    g = solver(prob, precision)
    I0 = g.get_intensity().astype(np.float64)
    e0, _, _ = g.gas()
    dt = 0.5 / oracle.Oracle(prob).positivity()
    g.run(3, dt)
    I = g.get_intensity().astype(np.float64)
    e, _, _ = g.gas()
    assert np.abs(I - I0).max() < tol * I0.max()
    assert np.abs(e - e0).max() < tol * e0.max()


def test_state_round_trip_refreshes_kappa_J():
    """kappa_J follows the gas temperature: a state saved and restored
    continues exactly as an uninterrupted run."""
    prob = _problem(CASES[0], 6, 8)
    dt = oracle.Oracle(prob).cfl_dt()
    a = solver(prob, "fp64")
    a.run(10, dt)
    ref = a.get_intensity()
    b = solver(prob, "fp64")
    b.run(5, dt)
    buf = b.get_state()
    b.run(3, dt)  # move away, then restore
    b.set_state(buf)
    b.run(5, dt)
    assert np.abs(b.get_intensity() - ref).max() == 0.0


def test_adjoint_refuses_temperature_dependent_opacity():
    import torch
    prob = make(n=(4, 4, 4), order=4)
    prob.beta_P, prob.beta_J, prob.T_ref = -3.0, 0.0, 1.0
    g = solver(prob, "fp64")
    N, A = prob.n_cells, prob.n_angles
    t = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.RTError) as err:
        g.adjoint_step(0.01, t(N, A), t(N), t(N, 3), t(N, A), t(N), t(N, 3), t(N), t(N))
    assert err.value.code == capi.RT_ERR_STATE
