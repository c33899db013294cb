"""CPU pins of the oracle's hand-written discrete adjoint.

The adjoint is checked against things it does not share code with: the
transpose identity <M d, l> = <d, M^T l> of the linear transport, and
central finite differences of the oracle's forward step (and of a multi-step
run) in every input direction: intensities, gas energy and momentum, and the
per-cell absorption opacities.
"""
import copy

import numpy as np
import pytest

import oracle
from tests._problems import make, randomise


def _problem(seed=3, moving=True):
    w = (0.2, -0.1, 0.15) if moving else None
    return randomise(make(n=(3, 3, 4), order=4, cbar=4.0, c=20.0, w=w), seed=seed, v_scale=0.05)


def test_transport_adjoint_is_transpose():
    prob = _problem()
    o = oracle.Oracle(prob)
    dt = 0.8 / o.positivity()
    rng = np.random.default_rng(0)
    d = rng.standard_normal((prob.n_cells, prob.n_angles))
    l = rng.standard_normal(d.shape)
    lhs = np.sum(o.transport(dt, d) * l)
    rhs = np.sum(d * o.transport_adjoint(dt, l))
    assert abs(lhs - rhs) < 1e-13 * np.sum(np.abs(d) * np.abs(l))


def _step_outputs(prob, dt, I, e, m):
    o = oracle.Oracle(prob)
    o.I[:] = I
    o.e[:] = e
    o.m[:] = m
    assert o.step(dt) == 0
    return o.I.copy(), o.e.copy(), o.m.copy()


@pytest.mark.parametrize("moving", [False, True])
def test_step_adjoint_matches_central_differences(moving):
    prob = _problem(seed=5, moving=moving)
    o = oracle.Oracle(prob)
    dt = 0.8 / o.positivity()
    N, A = prob.n_cells, prob.n_angles
    rng = np.random.default_rng(1)
    rI, re, rm = rng.standard_normal((N, A)), rng.standard_normal(N), rng.standard_normal((N, 3))

    def loss(I, e, m, p=prob):
        I1, e1, m1 = _step_outputs(p, dt, I, e, m)
        return np.sum(rI * I1) + np.sum(re * e1) + np.sum(rm * m1)

    I0, e0, m0 = o.I.copy(), o.e.copy(), o.m.copy()
    gP, gJ = np.zeros(N), np.zeros(N)
    lI, le, lm = o.adjoint_step(dt, I0, e0, m0, rI, re, rm, gP, gJ)

    def check(fd, ad):
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), abs(ad), 1e-30) + 1e-9 * (abs(fd) + 1e-30), (fd, ad)

    for trial in range(4):
        dI = rng.standard_normal((N, A)) * I0
        h = 1e-6
        fd = (loss(I0 + h * dI, e0, m0) - loss(I0 - h * dI, e0, m0)) / (2 * h)
        check(fd, np.sum(lI * dI))
        de = rng.standard_normal(N) * e0
        fd = (loss(I0, e0 + h * de, m0) - loss(I0, e0 - h * de, m0)) / (2 * h)
        check(fd, np.sum(le * de))
        dm = rng.standard_normal((N, 3)) * (np.abs(m0) + 1e-3 * prob.rho[:, None] * prob.c)
        fd = (loss(I0, e0, m0 + h * dm) - loss(I0, e0, m0 - h * dm)) / (2 * h)
        check(fd, np.sum(lm * dm))
    # per-cell opacities of interior cells
    interior = np.nonzero(prob.kind == 0)[0]
    for c in rng.choice(interior, size=min(6, interior.size), replace=False):
        for name, grad in (("kappa_P", gP), ("kappa_J", gJ)):
            h = 1e-6 * getattr(prob, name)[c]
            vals = []
            for sgn in (1, -1):
                p2 = copy.copy(prob)
                arr = getattr(prob, name).copy()
                arr[c] += sgn * h
                setattr(p2, name, arr)
                vals.append(loss(I0, e0, m0, p2))
            fd = (vals[0] - vals[1]) / (2 * h)
            check(fd, grad[c])


def _outflow_weights(prob):
    """dL/dI of the outgoing flux through +x: for every face from an interior
    cell into a +x boundary-layer cell, A 4 pi w_a cbar max(n_a . n_f, 0)."""
    m = prob.mesh
    ix = m.lattice_index()[0]
    bnd = (prob.kind == 1) & (ix == m.n[0] - 1)
    g = np.zeros((prob.n_cells, prob.n_angles))
    for f in range(m.n_faces):
        i, j = m.face_cells[f]
        for c, o, sgn in ((i, j, 1.0), (j, i, -1.0)):
            if prob.kind[c] != 1 and bnd[o]:
                mu = sgn * prob.dirs @ m.face_normal[f]
                g[c] += m.face_area[f] * 4 * np.pi * prob.weights * prob.cbar * np.maximum(mu, 0.0)
    return g


def test_multistep_gradient_matches_central_differences():
    """Outgoing flux through +x after K steps (the adjoint workload's loss on a
    small box): the chained adjoint gives dL/dkappa_a (kappa_P = kappa_J =
    kappa_a) and dL/dI^0 that central differences confirm."""
    from paper_2002_08377_gb300.inputs import adjoint
    prob = adjoint(n=6, steps=6)
    K = 6
    o = oracle.Oracle(prob)
    dt = o.cfl_dt()
    g = _outflow_weights(prob)
    assert g.sum() > 0

    def run(p):
        q = oracle.Oracle(p)
        states = []
        for _ in range(K):
            states.append((q.I.copy(), q.e.copy(), q.m.copy()))
            assert q.step(dt) == 0
        return q, states

    q, states = run(prob)
    L0 = np.sum(g * q.I)
    N = prob.n_cells
    lI, le, lm = g.copy(), np.zeros(N), np.zeros((N, 3))
    gP, gJ = np.zeros(N), np.zeros(N)
    for n in reversed(range(K)):
        I, e, m = states[n]
        lI, le, lm = q.adjoint_step(dt, I, e, m, lI, le, lm, gP, gJ)
    grad_kappa = gP + gJ
    rng = np.random.default_rng(7)
    interior = np.nonzero(prob.kind == 0)[0]
    # cells the outflow actually depends on
    cand = interior[np.abs(grad_kappa[interior]) > 1e-6 * np.abs(grad_kappa).max()]
    for c in rng.choice(cand, size=min(8, cand.size), replace=False):
        h = 1e-6 * prob.kappa_P[c]
        vals = []
        for sgn in (1, -1):
            p2 = copy.copy(prob)
            kp, kj = prob.kappa_P.copy(), prob.kappa_J.copy()
            kp[c] += sgn * h
            kj[c] += sgn * h
            p2.kappa_P, p2.kappa_J = kp, kj
            vals.append(np.sum(g * run(p2)[0].I))
        fd = (vals[0] - vals[1]) / (2 * h)
        # central differences carry the loss's round-off divided by h:
        # about 1e-16 * |L| * (operations) / 1e-6, below 1e-9 |L| here
        assert abs(fd - grad_kappa[c]) <= 1e-6 * abs(fd) + 1e-9 * abs(L0), (c, fd, grad_kappa[c])
    # initial intensity direction
    dI = rng.standard_normal((N, prob.n_angles)) * prob.initial_intensity()
    p_plus, p_minus = copy.copy(prob), copy.copy(prob)
    I_base = prob.initial_intensity()
    h = 1e-6
    p_plus.initial_intensity = lambda dtype=np.float64: I_base + h * dI
    p_minus.initial_intensity = lambda dtype=np.float64: I_base - h * dI
    fd = (np.sum(g * run(p_plus)[0].I) - np.sum(g * run(p_minus)[0].I)) / (2 * h)
    assert abs(fd - np.sum(lI * dI)) <= 1e-6 * abs(fd)
