"""CPU pins of the oracle's prescribed-radiation cells: boundary cells
(Sec. 2.4) and emitter cells (Sec. 2.5).

Both are source-only updates of a cell's intensities, so each test runs the
oracle's source step alone (no transport) on a 2x2x2 mesh whose cells are all
of one kind, and checks it against what the paper's equations fix:

* boundary cells follow the printed discrete relaxation
  I^{n+1} = I^n - (I^n - I0) min(dt/tau, 1); iterated n times this is
  I0 + (I - I0)(1 - dt/tau)^n, and as dt -> 0 it tends to the solution
  I0 + (I - I0) exp(-t/tau) of the relaxation equation dI/dt = -(I - I0)/tau;
* emitter cells integrate dI~/dt = Gamma cbar (rho kappa)_src (I_src - I~) in
  the comoving frame; with the gas frame fixed this has the closed-form
  solution I_src + (I~ - I_src) exp(-Gamma cbar (rho kappa)_src t), and the lab
  intensity is I = I~ / Gamma^4 (Sec. 2.3 transformation, Gamma = 1 - v.n/c at
  first order, gamma (1 - v.n/c) to all orders).  The implicit update is first
  order in time, so substeps converge to that solution at first order, and
  I = I_src / Gamma^4 is its fixed point.

The energy the radiation loses in these cells goes to the cell's external
tally, (c/cbar) 4 pi sum_a w_a (I_a - I'_a) (Eq. gas1 with the cell's gas held
fixed), which the tests also check against the closed forms.
"""
import numpy as np
import pytest

import oracle
from tests._problems import make


def _cells(kind, order=4, v=(0.0, 0.0, 0.0), boost=0, seed=3, c=10.0, cbar=10.0):
    """2x2x2 jittered mesh, every cell of the given kind, random anisotropic
    initial intensities; the gas frame velocity v (emitters only read it)."""
    prob = make(n=(2, 2, 2), order=order, cbar=cbar, c=c, v=v)
    rng = np.random.default_rng(seed)
    N, A = prob.n_cells, prob.n_angles
    prob.kind = np.full(N, kind, np.uint8)
    I = rng.uniform(0.1, 2.0, (N, A))
    prob.initial_intensity = lambda dtype=np.float64, _I=I: np.ascontiguousarray(_I.astype(dtype))
    prob.boost = boost
    return prob, I, rng


def _source_steps(o, dt, n, I):
    """n source-only steps of the oracle from I (gas and tallies in o)."""
    cur = np.array(I, dtype=np.float64, copy=True)
    for _ in range(n):
        st, cur = o.source(dt, cur)
        assert st == oracle.ORC_OK
    return cur


# ------------------------------------------------------------- boundary cells
@pytest.mark.parametrize("ratio", [4.0, 2.5])
def test_boundary_partial_relaxation_iterates_printed_scheme(ratio):
    """tau = ratio * dt > dt: n steps give I0 + (I - I0)(1 - dt/tau)^n to
    round-off (the printed discrete relaxation, iterated), for per-cell tau
    and per-row I0; the gas is untouched and the tally holds the energy the
    radiation lost."""
    prob, I, rng = _cells(1)
    N, A = prob.n_cells, prob.n_angles
    dt = 1e-3
    prob.tau = dt * ratio * rng.uniform(1.0, 3.0, N)
    prob.I0 = rng.uniform(0.0, 1.5, (2, A))
    prob.bc_row = (np.arange(N) % 2).astype(np.int32)
    o = oracle.Oracle(prob)
    e0, m0 = o.e.copy(), o.m.copy()
    n = 7
    out = _source_steps(o, dt, n, I)
    I0 = prob.I0[prob.bc_row]
    keep = (1.0 - dt / prob.tau)[:, None] ** n
    want = I0 + (I - I0) * keep
    assert np.abs(out - want).max() <= 1e-14 * np.abs(want).max()
    assert np.array_equal(o.e, e0) and np.array_equal(o.m, m0)
    lost = prob.c / prob.cbar * 4 * np.pi * ((I - want) @ prob.weights)
    assert np.abs(o.ext[:, 0] - lost).max() <= 1e-13 * np.abs(lost).max()


def test_boundary_relaxation_converges_to_exponential():
    """At fixed tau, substeps converge at first order in dt to the solution
    I0 + (I - I0) exp(-t/tau) of dI/dt = -(I - I0)/tau (Sec. 2.4), so a
    factor dt/tau inverted or the min(dt/tau, 1) cap applied below tau
    would fail."""
    prob, I, rng = _cells(1, seed=5)
    N, A = prob.n_cells, prob.n_angles
    t_end = 0.02
    prob.tau = rng.uniform(0.01, 0.04, N)
    prob.I0 = rng.uniform(0.0, 1.5, (1, A))
    prob.bc_row = np.zeros(N, np.int32)
    exact = prob.I0[0] + (I - prob.I0[0]) * np.exp(-t_end / prob.tau)[:, None]
    errs = []
    for n in (16, 32, 64, 128):
        o = oracle.Oracle(prob)
        out = _source_steps(o, t_end / n, n, I)
        errs.append(np.abs(out - exact).max())
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 1.0) < 0.08), (errs, slopes)
    assert errs[-1] < 1e-2 * np.abs(exact).max()


def test_boundary_short_tau_pins_I0():
    """tau <= dt: one step sets I = I0 (min(dt/tau, 1) = 1), to the rounding
    of I - (I - I0)."""
    prob, I, rng = _cells(1, seed=9)
    N, A = prob.n_cells, prob.n_angles
    dt = 1e-3
    prob.tau = np.where(np.arange(N) % 2 == 0, 0.0, dt * rng.uniform(0.2, 1.0, N))
    prob.I0 = rng.uniform(0.0, 1.5, (1, A))
    prob.bc_row = np.zeros(N, np.int32)
    o = oracle.Oracle(prob)
    out = _source_steps(o, dt, 1, I)
    assert np.abs(out - prob.I0[0]).max() <= 4e-16 * max(np.abs(I).max(), np.abs(prob.I0).max())


# -------------------------------------------------------------- emitter cells
def _gamma(prob, v, boost):
    n = prob.dirs
    G = 1.0 - (n @ np.asarray(v, float)) / prob.c
    if boost:
        G = G / np.sqrt(1.0 - np.dot(v, v) / prob.c ** 2)
    return G


@pytest.mark.parametrize("v,boost", [((0.0, 0.0, 0.0), 0), ((2.0, -1.0, 1.5), 0),
                                     ((3.0, 2.0, -1.0), 1)])
def test_emitter_converges_to_comoving_exponential(v, boost):
    """Emitter substeps converge at first order to the closed-form solution of
    dI~/dt = Gamma cbar (rho kappa)_src (I_src - I~) with lab I = I~/Gamma^4
    (Sec. 2.5 with the Sec. 2.3 transformation).  A Gamma^3 back-transform, a
    missing Gamma in the rate, or c in place of cbar all move the limit."""
    prob, I, rng = _cells(2, v=v, boost=boost, c=10.0, cbar=5.0)
    N = prob.n_cells
    prob.emit_rate = rng.uniform(5.0, 20.0, N)
    prob.I_src = rng.uniform(0.5, 2.0, N)
    G = _gamma(prob, v, boost)[None, :]
    t_end = 0.01
    It0 = G ** 4 * I
    rate = G * prob.cbar * prob.emit_rate[:, None]
    exact = (prob.I_src[:, None] + (It0 - prob.I_src[:, None]) * np.exp(-rate * t_end)) / G ** 4
    errs = []
    for n in (16, 32, 64, 128):
        o = oracle.Oracle(prob)
        out = _source_steps(o, t_end / n, n, I)
        errs.append(np.abs(out - exact).max())
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 1.0) < 0.08), (errs, slopes)
    assert errs[-1] < 5e-3 * np.abs(exact).max()


@pytest.mark.parametrize("v,boost", [((2.0, -1.0, 1.5), 0), ((3.0, 2.0, -1.0), 1)])
def test_emitter_moving_fixed_point(v, boost):
    """Lab I = I_src / Gamma^4 (isotropic I_src in the comoving frame) is a
    fixed point of the emitter update at any dt; the gas reservoir and its
    frame stay untouched and the tally holds what the radiation lost
    (nothing here, to round-off)."""
    prob, _, rng = _cells(2, v=v, boost=boost)
    N = prob.n_cells
    prob.emit_rate = rng.uniform(5.0, 20.0, N)
    prob.I_src = rng.uniform(0.5, 2.0, N)
    G = _gamma(prob, v, boost)[None, :]
    I = prob.I_src[:, None] / G ** 4
    o = oracle.Oracle(prob)
    e0, m0 = o.e.copy(), o.m.copy()
    out = _source_steps(o, 0.05, 3, I)
    assert np.abs(out / I - 1.0).max() < 1e-13
    assert np.array_equal(o.e, e0) and np.array_equal(o.m, m0)
    assert np.abs(o.ext[:, 0]).max() < 1e-13 * np.abs(I).max() * prob.c / prob.cbar * 4 * np.pi


def test_emitter_at_rest_iterates_backward_euler():
    """v = 0: n steps of the implicit emitter update equal I_src + (I - I_src)
    (1 + y)^-n with y = dt cbar (rho kappa)_src, to round-off, and the tally
    equals the energy gained (negative: the emitter injects)."""
    prob, I, rng = _cells(2, seed=13)
    N = prob.n_cells
    prob.emit_rate = rng.uniform(1.0, 50.0, N)
    prob.I_src = rng.uniform(0.5, 4.0, N)
    dt, n = 3e-3, 9
    o = oracle.Oracle(prob)
    out = _source_steps(o, dt, n, I)
    y = dt * prob.cbar * prob.emit_rate
    want = prob.I_src[:, None] + (I - prob.I_src[:, None]) * ((1.0 + y) ** -n)[:, None]
    assert np.abs(out - want).max() <= 1e-14 * np.abs(want).max()
    lost = prob.c / prob.cbar * 4 * np.pi * ((I - want) @ prob.weights)
    assert np.abs(o.ext[:, 0] - lost).max() <= 1e-13 * np.abs(lost).max()
