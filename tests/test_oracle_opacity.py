"""CPU pins of the oracle's temperature-dependent opacities.

Sec. 2.3 solves the temperature equation by Newton-Raphson when the opacity
depends on temperature.  The reading: kappa_P(T) = kappa_P (T/T_ref)^beta_P is
taken at T^{n+1}, inside the solve, so the equation becomes
alpha T^(4 + beta_P) + rho c_v T = g; kappa_J(T) = kappa_J (T/T_ref)^beta_J is
taken at the start of the step, so the angular sums keep their closed form.
Pins: the power-law root against an independent root finder and a closed
form, the equilibrium of a medium whose two opacities share the exponent, and
conservation.  (The subcycled-ODE pin in tests/test_oracle_pins.py integrates
the source equations with both opacities at the running temperature.)
"""
import mpmath
import numpy as np
import pytest

import oracle
from tests._problems import make, randomise


def test_power_newton_matches_mpmath_and_closed_forms():
    """Root of alpha T^k + beta T = g within 4 ulp of a 60-digit bisection for
    k from 1 to 7.5 over 12 decades of coefficients; k = 1 is the closed form
    g / (alpha + beta), k = 4 the quartic solver's root."""
    mpmath.mp.dps = 60
    rng = np.random.default_rng(5)
    for _ in range(120):
        k = float(rng.choice([1.0, 1.5, 2.5, 4.0, 7.5]))
        alpha, beta, g = 10.0 ** rng.uniform(-6, 6, 3)
        st, T, it = oracle.newton_power(alpha, k, beta, g)
        assert st == oracle.ORC_OK and it <= 64
        A, B, G, K = mpmath.mpf(alpha), mpmath.mpf(beta), mpmath.mpf(g), mpmath.mpf(k)
        lo, hi = mpmath.mpf(0), min(G / B, (G / A) ** (1 / K))
        for _ in range(220):
            mid = (lo + hi) / 2
            if A * mid ** K + B * mid - G > 0:
                hi = mid
            else:
                lo = mid
        ref = float((lo + hi) / 2)
        assert abs(T - ref) <= 4 * np.spacing(ref), (k, alpha, beta, g, T, ref)
        if k == 1.0:
            assert abs(T - g / (alpha + beta)) <= 4 * np.spacing(T)
        if k == 4.0:
            _, T4, _ = oracle.newton(alpha, beta, g)
            assert abs(T - T4) <= 4 * np.spacing(T4)


@pytest.mark.parametrize("betas,fixed", [((1.5, 1.5), True), ((-3.0, -3.0), True),
                                         ((2.0, -1.0), False)])
def test_equilibrium_with_temperature_dependent_opacity(betas, fixed):
    """A uniform medium at T = 1.3 with I = a T^4 / 4 pi and T_ref = 0.6: with
    beta_P = beta_J both opacities are equal at every temperature, so the
    medium stays in equilibrium (to 1e-12 over three steps); with different
    exponents kappa_P(T) != kappa_J(T) and it moves."""
    T = 1.3
    prob = make(n=(3, 4, 3), order=6, cbar=5.0, c=20.0, T=T, kP=2.0, kJ=2.0, kS=0.4)
    prob.beta_P, prob.beta_J = betas
    prob.T_ref = 0.6
    o = oracle.Oracle(prob)
    I0, e0 = o.I.copy(), o.e.copy()
    dt = 0.5 / o.positivity()
    for _ in range(3):
        assert o.step(dt) == oracle.ORC_OK
    dev = max(np.abs(o.I - I0).max() / I0.max(), np.abs(o.e - e0).max() / e0.max())
    if fixed:
        assert dev < 1e-12
    else:
        assert dev > 1e-4


def test_temperature_dependent_opacity_conserves_energy_and_momentum():
    prob = randomise(make(n=(4, 3, 5), order=6, cbar=10.0, c=100.0, w=(0.3, 0.1, 0.0)), seed=9)
    prob.beta_P, prob.beta_J, prob.T_ref = -3.0, 1.5, 0.8
    o = oracle.Oracle(prob)
    dt = 0.9 / o.positivity()
    t0 = o.totals()
    assert o.run(20, dt) == oracle.ORC_OK
    t1 = o.totals()
    assert abs(t1[12] - t0[12]) < 1e-13 * abs(t0[12])
    scale = np.abs(t0[3:12]).sum() + np.abs(t1[3:12]).sum()
    assert np.abs(t1[13:16] - t0[13:16]).max() < 1e-13 * scale
    assert abs(t1[0] - t0[0]) > 1e-6 * abs(t0[12])
