"""GPU parity of the comoving transformation to all orders in v/c
(rt_params.boost = 1, Gamma = gamma (1 - v.n/c), Sec. 2.3), through the C ABI
against the FP64 oracle: RT_FP64 per intensity to a relative 1e-12, RT_FP32
in L1 of E_r to 1e-5 with total energy conserved to 1e-6."""
import numpy as np
import pytest

import oracle
from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from tests._problems import make, randomise
from tests.test_gpu_parity import check_fp32, check_fp64, rel_err, solver
from tests.test_oracle_boost import _moving_equilibrium

pytestmark = pytest.mark.gpu

FP32_ENERGY = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()
    capi.load()


def _boosted(n, order, seed, w=None):
    """Random opacities, boundary / emitter cells, scattering, |v|/c up to
    0.43 (gamma up to 1.11), c != cbar."""
    prob = randomise(make(n=n, order=order, cbar=10.0, c=100.0, w=w), seed=seed, v_scale=0.25)
    prob.boost = 1
    return prob


@pytest.mark.parametrize("order,n", [(6, (9, 7, 5)), (8, (4, 3, 5))])
@pytest.mark.parametrize("w", [None, (0.3, -0.1, 0.2)])
def test_fp64_all_orders_random_problem(order, n, w):
    prob = _boosted(n, order, 5, w)
    o = oracle.Oracle(prob)
    g = solver(prob, "fp64")
    dt = o.cfl_dt()
    assert o.run(30, dt) == oracle.ORC_OK
    g.run(30, dt)
    check_fp64(o, g)
    # the transformation to all orders changed the result
    o1 = oracle.Oracle(_boosted(n, order, 5, w))
    o1.p.boost_all_orders = 0
    assert o1.run(30, dt) == oracle.ORC_OK
    assert rel_err(o1.I, o.I) > 1e-6


@pytest.mark.parametrize("order", [6, 8])
def test_fp32_all_orders_random_problem(order):
    prob = _boosted((9, 7, 5), order, 6, (0.3, -0.1, 0.2))
    o = oracle.Oracle(prob)
    g = solver(prob, "fp32")
    t0 = g.totals()
    dt = o.cfl_dt()
    assert o.run(30, dt) == oracle.ORC_OK
    g.run(30, dt)
    check_fp32(o, g)
    t1 = g.totals()
    assert abs(t1[12] - t0[12]) < FP32_ENERGY * abs(t0[12])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_moving_equilibrium_stays_on_the_gpu(precision, tol):
    """The oracle's fixed point at |v| = c/2: I = B / Gamma^4 with the
    all-orders Gamma is left unchanged by three GPU steps."""
    prob = _moving_equilibrium(1)
    g = solver(prob, precision)
    I0 = g.get_intensity().astype(np.float64)
    e0, m0, _ = g.gas()
    dt = 0.5 / oracle.Oracle(prob).positivity()
    g.run(3, dt)
    I = g.get_intensity().astype(np.float64)
    e, m, _ = g.gas()
    assert np.abs(I - I0).max() < tol * I0.max()
    assert np.abs(e - e0).max() < tol * e0.max()


def test_van_leer_all_orders_fp64():
    prob = _boosted((6, 5, 7), 6, 7, (0.2, -0.1, 0.15))
    prob.integrator = capi.RT_VAN_LEER
    o = oracle.Oracle(prob)
    g = solver(prob, "fp64")
    dt = 0.5 / o.positivity()
    assert o.run(20, dt) == oracle.ORC_OK
    g.run(20, dt)
    check_fp64(o, g)


def test_adjoint_refuses_a_boosted_state():
    import torch
    prob = make(n=(4, 4, 4), order=4)
    prob.boost = 1
    g = solver(prob, "fp64")
    N, A = prob.n_cells, prob.n_angles
    t = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.RTError) as err:
        g.adjoint_step(0.01, t(N, A), t(N), t(N, 3), t(N, A), t(N), t(N, 3), t(N), t(N))
    assert err.value.code == capi.RT_ERR_STATE

