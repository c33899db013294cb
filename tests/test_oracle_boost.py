"""CPU pins of the oracle's comoving transformation to all orders in v/c.

Sec. 2.3 defines the lab-to-comoving frequency ratio as Gamma = gamma
(1 - v . n / c) with gamma the Lorentz factor, and notes that boosting to the
fluid frame and back makes the source step accurate to all orders in v/c.
The first-order problem takes gamma = 1; the flag `boost` takes the full
factor.  Besides the subcycled-ODE pin (tests/test_oracle_pins.py), these
check that a medium in equilibrium stays in equilibrium when it moves (its
lab intensities are the comoving Planck intensity divided by Gamma^4, with
the Gamma of the problem's order) and that the lab-frame exchange conserves
energy and momentum at relativistic speeds.
"""
import numpy as np
import pytest

import oracle
from tests._problems import make, randomise


def _moving_equilibrium(boost, beta=0.5, T=1.3):
    rng = np.random.default_rng(3)
    vhat = rng.standard_normal(3)
    vhat /= np.linalg.norm(vhat)
    c = 20.0
    v = beta * c * vhat
    prob = make(n=(4, 4, 4), order=6, cbar=5.0, c=c, T=T, v=v, kP=2.0, kJ=2.0, kS=0.7)
    prob.boost = boost
    gam = 1 / np.sqrt(1 - beta ** 2) if boost else 1.0
    G = gam * (1 - prob.dirs @ v / c)
    B = prob.a_rad * T ** 4 / (4 * np.pi)
    prob.J0 = np.ones(prob.n_cells)
    prob.q0 = B / G ** 4
    return prob


@pytest.mark.parametrize("boost", [0, 1])
def test_moving_equilibrium_is_a_fixed_point(boost):
    """A uniform medium at temperature T moving at |v| = c/2 (gamma = 1.155)
    with lab intensities B(T) / Gamma^4, Gamma of the problem's order, is left
    unchanged by a full step (transport, absorption, emission, scattering and
    the gas exchange); the same field with the other order's Gamma is not."""
    prob = _moving_equilibrium(boost)
    o = oracle.Oracle(prob)
    I0, e0, m0 = o.I.copy(), o.e.copy(), o.m.copy()
    dt = 0.5 / o.positivity()
    for _ in range(3):
        assert o.step(dt) == oracle.ORC_OK
    assert np.abs(o.I - I0).max() < 1e-12 * I0.max()
    assert np.abs(o.e - e0).max() < 1e-12 * e0.max()
    assert np.abs(o.m - m0).max() < 1e-12 * np.abs(m0).max()
    other = _moving_equilibrium(boost)
    other.boost = 1 - boost
    o2 = oracle.Oracle(other)
    assert o2.step(dt) == oracle.ORC_OK
    assert np.abs(o2.I - I0).max() > 1e-3 * I0.max()


def test_all_orders_conserves_energy_and_momentum():
    """Sec. 2.3.1 totals with Gamma to all orders at |v|/c up to 0.43: the
    exchange is formed from lab-frame moments, so E_gas + (c/cbar) E_r and
    rho v + F_r/(c cbar) (with the boundary / emitter tallies) stay constant
    to round-off on a moving mesh with scattering."""
    prob = randomise(make(n=(4, 3, 5), order=6, cbar=10.0, c=100.0, w=(0.3, 0.1, 0.0)), seed=9,
                     v_scale=0.25)
    prob.boost = 1
    o = oracle.Oracle(prob)
    dt = 0.9 / o.positivity()
    t0 = o.totals()
    assert o.run(20, dt) == oracle.ORC_OK
    t1 = o.totals()
    assert abs(t1[12] - t0[12]) < 1e-13 * abs(t0[12])
    scale = np.abs(t0[3:12]).sum() + np.abs(t1[3:12]).sum()
    assert np.abs(t1[13:16] - t0[13:16]).max() < 1e-13 * scale
    assert abs(t1[0] - t0[0]) > 1e-6 * abs(t0[12])


def test_adjoint_refuses_the_all_orders_transformation():
    prob = make(n=(3, 3, 3), order=4)
    prob.boost = 1
    o = oracle.Oracle(prob)
    N, A = prob.n_cells, prob.n_angles
    z = np.zeros(N)
    with pytest.raises(ValueError):
        o.adjoint_step(0.01, o.I, o.e, o.m, np.ones((N, A)), z, np.zeros((N, 3)), z.copy(), z.copy())

