"""CPU pins of the oracle's frequency groups (Sec. 2.3: "multiple independent
frequency groups" that couple only through the temperature).

Group j holds its own intensities on the same angles, its own opacities and
a group weight W_j; the temperature equation sums the groups with W_j and the
gas exchange uses the weights W_j w_a.  Pins: identical groups reproduce the
grey step, a medium in equilibrium stays there with unequal group opacities,
a transparent group is untouched by the source step, the implicit update
converges to a subcycled RK4 integration of the groups' source equations at
first order, and energy and momentum are conserved.
"""
import numpy as np
import pytest

import oracle
from tests._problems import grouped, make, randomise


def test_identical_groups_reproduce_the_grey_step():
    base = lambda: randomise(make(n=(4, 3, 5), order=6, cbar=10.0, c=100.0, w=(0.3, 0.1, 0.0)),
                             seed=9)
    grey = oracle.Oracle(base())
    grp = oracle.Oracle(grouped(base(), (0.3, 0.7)))
    dt = 0.9 / grey.positivity()
    assert grey.run(10, dt) == oracle.ORC_OK
    assert grp.run(10, dt) == oracle.ORC_OK
    A = grey.A
    for j in range(2):
        assert np.abs(grp.I[:, j * A:(j + 1) * A] - grey.I).max() < 1e-13 * grey.I.max()
    assert np.abs(grp.e - grey.e).max() < 1e-13 * grey.e.max()
    assert np.abs(grp.m - grey.m).max() < 1e-13 * (np.abs(grey.m).max() + 1.0)


def test_equilibrium_with_unequal_group_opacities():
    T = 1.3
    prob = grouped(make(n=(3, 4, 3), order=6, cbar=5.0, c=20.0, T=T, kP=2.0, kJ=2.0, kS=0.4),
                   (0.2, 0.5, 0.3), scale_P=(0.1, 1.0, 8.0), scale_J=(0.1, 1.0, 8.0),
                   scale_S=(3.0, 0.0, 1.0))
    o = oracle.Oracle(prob)
    I0, e0 = o.I.copy(), o.e.copy()
    dt = 0.5 / o.positivity()
    for _ in range(3):
        assert o.step(dt) == oracle.ORC_OK
    assert np.abs(o.I - I0).max() < 1e-12 * I0.max()
    assert np.abs(o.e - e0).max() < 1e-12 * e0.max()


def test_transparent_group_is_untouched_by_the_source():
    prob = grouped(randomise(make(n=(3, 3, 3), order=6, cbar=5.0, c=20.0), seed=3, kinds=False),
                   (0.6, 0.4), scale_P=(1.0, 0.0), scale_J=(1.0, 0.0), scale_S=(1.0, 0.0),
                   I_group=(1.0, 0.5))
    o = oracle.Oracle(prob)
    A = o.A // 2
    st, I1 = o.source(0.05, o.I)
    assert st == oracle.ORC_OK
    # (to rounding: the group goes to the moving frame and back, Gamma^4 I / Gamma^4)
    assert np.abs(I1[:, A:] - o.I[:, A:]).max() < 1e-15 * o.I[:, A:].max()
    assert np.abs(I1[:, :A] - o.I[:, :A]).max() > 1e-3 * o.I.max()


def _ode_groups(prob, c, I0, dt, steps):
    """RK4 of the groups' comoving source equations (Eq. com radiative source
    per group j, Eq. com rad thermal with the group weights W_j) for one cell,
    frame velocity frozen."""
    G, W = prob.n_groups, prob.group_w
    d, w = prob.dirs, prob.weights
    rho = prob.rho[c]
    v = prob.m[c] / rho
    Gam = 1 - d @ v / prob.c
    wc = w / Gam ** 2
    wc /= wc.sum()
    rcv = rho * prob.r_gas / (prob.gamma_gas - 1)
    T0 = (prob.e[c] - 0.5 * np.sum(prob.m[c] ** 2) / rho) / rcv
    kP, kJ, kS = prob.kappa_P[c], prob.kappa_J[c], prob.kappa_s[c]
    A = d.shape[0]
    y = np.concatenate([np.concatenate([Gam ** 4 * I0[j * A:(j + 1) * A] for j in range(G)]), [T0]])

    def f(y):
        T = y[-1]
        out, heat = [], 0.0
        for j in range(G):
            It = y[j * A:(j + 1) * A]
            J = wc @ It
            out.append(Gam * prob.cbar * rho * (kP[j] * prob.a_rad * T ** 4 / (4 * np.pi)
                                                + kS[j] * J - (kJ[j] + kS[j]) * It))
            heat += W[j] * prob.c * rho * (kP[j] * prob.a_rad * T ** 4 - 4 * np.pi * kJ[j] * J)
        return np.concatenate(out + [[-heat / rcv]])

    h = dt / steps
    for _ in range(steps):
        k1 = f(y); k2 = f(y + h / 2 * k1); k3 = f(y + h / 2 * k2); k4 = f(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return np.concatenate([y[j * A:(j + 1) * A] / Gam ** 4 for j in range(G)]), y[-1]


def test_groups_converge_to_subcycled_explicit():
    prob = grouped(randomise(make(n=(2, 2, 2), order=4, cbar=5.0, c=50.0), seed=4, kinds=False),
                   (0.2, 0.5, 0.3), scale_P=(0.3, 1.0, 3.0), scale_J=(0.5, 1.0, 2.0),
                   scale_S=(2.0, 0.5, 0.0), I_group=(1.5, 1.0, 0.4))
    I_start = prob.initial_intensity()
    dt = 0.02
    ref = [_ode_groups(prob, c, I_start[c], dt, 4000) for c in range(prob.n_cells)]
    errs = []
    for nsub in (8, 16, 32):
        o = oracle.Oracle(prob)
        I = I_start.copy()
        for _ in range(nsub):
            st, I = o.source(dt / nsub, I)
            assert st == oracle.ORC_OK
        errs.append(max(np.abs(I[c] - ref[c][0]).max() / np.abs(ref[c][0]).max()
                        for c in range(prob.n_cells)))
    assert errs[-1] < 0.05
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


def test_groups_conserve_energy_and_momentum():
    prob = grouped(randomise(make(n=(4, 3, 5), order=6, cbar=10.0, c=100.0, w=(0.3, 0.1, 0.0)),
                             seed=9), (0.25, 0.75), scale_P=(0.2, 4.0), scale_J=(0.3, 2.0),
                   scale_S=(1.0, 0.1), I_group=(2.0, 0.5))
    o = oracle.Oracle(prob)
    dt = 0.9 / o.positivity()
    t0 = o.totals()
    assert o.run(20, dt) == oracle.ORC_OK
    t1 = o.totals()
    assert abs(t1[12] - t0[12]) < 1e-13 * abs(t0[12])
    scale = np.abs(t0[3:12]).sum() + np.abs(t1[3:12]).sum()
    assert np.abs(t1[13:16] - t0[13:16]).max() < 1e-13 * scale
    assert abs(t1[0] - t0[0]) > 1e-6 * abs(t0[12])
