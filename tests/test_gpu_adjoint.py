"""GPU adjoint: rt_adjoint_step and the autograd run against the oracle's
discrete adjoint and against central differences of the oracle's forward
run (the adjoint workload: outgoing flux through +x, gradient with respect
to the per-cell absorption opacity and the initial intensities)."""
import copy

import numpy as np
import pytest

import oracle
from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from paper_2002_08377_gb300.autograd import outflow_weights, run
from paper_2002_08377_gb300.inputs import adjoint
from tests._problems import make, randomise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()
    capi.load()


def _solver(prob, precision):
    from paper_2002_08377_gb300.solver import RTSolver
    return RTSolver.from_problem(prob, precision)


def _gas(prob):
    return {"rho": prob.rho, "e": prob.e, "m": prob.m, "kappa_s": prob.kappa_s}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
@pytest.mark.parametrize("moving", [False, True])
def test_adjoint_step_matches_oracle(precision, tol, moving):
    import torch
    w = (0.2, -0.1, 0.15) if moving else None
    prob = randomise(make(n=(6, 5, 7), order=6, cbar=4.0, c=20.0, w=w), seed=9, v_scale=0.05)
    o = oracle.Oracle(prob)
    dt = 0.8 / o.positivity()
    assert o.run(2, dt) == 0  # a non-trivial state (moving gas, filled tallies)
    N, A = prob.n_cells, prob.n_angles
    rng = np.random.default_rng(4)
    lI1, le1, lm1 = rng.standard_normal((N, A)), rng.standard_normal(N), rng.standard_normal((N, 3))
    gP_o, gJ_o = np.zeros(N), np.zeros(N)
    lI_o, le_o, lm_o = o.adjoint_step(dt, o.I, o.e, o.m, lI1, le1, lm1, gP_o, gJ_o)

    g = _solver(prob, precision)
    dev = lambda x: torch.tensor(x, device="cuda")
    gP, gJ = torch.zeros(N, dtype=torch.float64, device="cuda"), torch.zeros(N, dtype=torch.float64,
                                                                             device="cuda")
    lI, le, lm = g.adjoint_step(dt, dev(o.I), dev(o.e), dev(o.m), dev(lI1), dev(le1), dev(lm1), gP, gJ)

    def close(x, y):
        x = x.detach().cpu().numpy().astype(np.float64)
        assert np.abs(x - y).max() <= tol * np.abs(y).max(), (np.abs(x - y).max(), np.abs(y).max())

    close(lI, lI_o)
    close(le, le_o)
    close(lm, lm_o)
    close(gP, gP_o)
    close(gJ, gJ_o)


def test_outflow_weights_definition():
    """The package's outgoing-flux weights equal a plain loop over faces."""
    prob = adjoint(n=6, steps=2)
    g = outflow_weights(prob)
    m = prob.mesh
    ix = m.lattice_index()[0]
    bnd = (prob.kind == 1) & (ix == m.n[0] - 1)
    ref = np.zeros_like(g)
    for f in range(m.n_faces):
        i, j = m.face_cells[f]
        for c, o, sg in ((i, j, 1.0), (j, i, -1.0)):
            if prob.kind[c] != 1 and bnd[o]:
                mu = sg * prob.dirs @ m.face_normal[f]
                ref[c] += m.face_area[f] * 4 * np.pi * prob.weights * prob.cbar * np.maximum(mu, 0)
    assert np.allclose(g, ref, rtol=1e-14, atol=0) and g.sum() > 0


def _oracle_loss_and_grad(prob, dt, K, g):
    o = oracle.Oracle(prob)
    states = []
    for _ in range(K):
        states.append((o.I.copy(), o.e.copy(), o.m.copy()))
        assert o.step(dt) == 0
    L = float(np.sum(g * o.I))
    N = prob.n_cells
    lI, le, lm = g.copy(), np.zeros(N), np.zeros((N, 3))
    gP, gJ = np.zeros(N), np.zeros(N)
    for n in reversed(range(K)):
        I, e, m = states[n]
        lI, le, lm = o.adjoint_step(dt, I, e, m, lI, le, lm, gP, gJ)
    return L, gP + gJ, lI


def _oracle_loss(prob, dt, K, g, kappa=None, I0=None):
    p = copy.copy(prob)
    if kappa is not None:
        p.kappa_P, p.kappa_J = kappa.copy(), kappa.copy()
    if I0 is not None:
        p.initial_intensity = lambda dtype=np.float64, _I=I0: _I.astype(dtype)
    o = oracle.Oracle(p)
    for _ in range(K):
        assert o.step(dt) == 0
    return float(np.sum(g * o.I))


def _autograd(prob, precision, dt, K, every, g):
    import torch
    s = _solver(prob, precision)
    I0 = torch.tensor(prob.initial_intensity(s.dtype), device="cuda", requires_grad=True)
    kap = torch.tensor(prob.kappa_P, dtype=torch.float64, requires_grad=True)
    out = run(s, I0, kap, _gas(prob), K, dt, every)
    L = (out.double() * torch.tensor(g, device="cuda")).sum()
    L.backward()
    res = (float(L.detach()), kap.grad.cpu().numpy(), I0.grad.double().cpu().numpy())
    s.close()
    return res


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-3)])
def test_autograd_gradient_matches_oracle_adjoint(precision, tol):
    """Adjoint workload on a 16^3 box, 16 steps, checkpoints every 4."""
    prob = adjoint(n=16, steps=16)
    dt = prob.cfl_dt()
    g = outflow_weights(prob)
    L_o, gk_o, gI_o = _oracle_loss_and_grad(prob, dt, 16, g)
    L, gk, gI = _autograd(prob, precision, dt, 16, 4, g)
    assert abs(L - L_o) <= tol * abs(L_o)
    assert np.abs(gk - gk_o).max() <= tol * np.abs(gk_o).max()
    assert np.abs(gI - gI_o).max() <= tol * np.abs(gI_o).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_workload_full_size_against_finite_differences(precision):
    """The adjoint workload at full size (64^3 cells, 48 angles, 64 steps,
    checkpoint every 8): the GPU gradient with respect to kappa_a, projected on
    a random direction supported on 32 random interior cells, matches central
    differences of the FP64 oracle to 1e-4 relative."""
    prob = adjoint()
    K = 64
    dt = prob.cfl_dt()
    g = outflow_weights(prob)
    L, gk, _ = _autograd(prob, precision, dt, K, 8, g)
    rng = np.random.default_rng(11)
    interior = np.nonzero(prob.kind == 0)[0]
    # cells the loss depends on measurably
    cand = interior[np.abs(gk[interior]) > 1e-3 * np.abs(gk).max()]
    cells = rng.choice(cand, size=32, replace=False)
    d = np.zeros(prob.n_cells)
    d[cells] = rng.uniform(0.5, 1.5, 32) * prob.kappa_P[cells]
    h = 1e-5
    Lp = _oracle_loss(prob, dt, K, g, kappa=prob.kappa_P + h * d)
    Lm = _oracle_loss(prob, dt, K, g, kappa=prob.kappa_P - h * d)
    fd = (Lp - Lm) / (2 * h)
    ad = float(np.sum(gk * d))
    assert abs(ad - fd) <= 1e-4 * abs(fd), (ad, fd)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_gradient_per_cell_against_oracle_differences(precision):
    """The full-size adjoint workload (64^3 cells, 48 angles, 64 steps,
    checkpoint every 8): the GPU gradient of the outflow loss, cell by cell,
    against central differences of the FP64 oracle stored in
    tests/golden/adjoint_fd_64.json (written by make_adjoint_fd.py, which
    calls only the oracle): dL/dkappa_a at 32 random interior cells and
    dL/dI0 at 16 random (cell, angle) entries, each to a relative 1e-4 with a
    floor of 1e-3 of the largest derivative (FP64).  FP32 gradients carry an
    absolute error set by float rounding of the 64 reverse steps' sums (each
    cell's dL/dkappa is a sum of absorption and emission terms of opposite
    sign, over 48 angles and 64 steps): measured up to 1.6e-6 of the largest
    derivative, so its floor is 5e-2 of the largest (an absolute 5e-6 of it,
    about 80 float ulps); above the floor the relative bar is the same 1e-4."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "adjoint_fd_64.json")
    gold = json.load(open(path))
    prob = adjoint(n=gold["n"], steps=gold["steps"])
    dt = prob.cfl_dt()
    assert abs(dt / gold["dt"] - 1) < 1e-12
    g = outflow_weights(prob)
    L, gk, gI = _autograd(prob, precision, dt, gold["steps"], 8, g)
    assert abs(L / gold["loss"] - 1) < (1e-12 if precision == "fp64" else 1e-5)
    floor = 1e-3 if precision == "fp64" else 5e-2
    fk = gold["max_abs_dL_dkappa"] * floor
    fi = gold["max_abs_dL_dI0"] * floor
    rel_k = [abs(gk[e["cell"]] - e["fd"]) / max(abs(e["fd"]), fk) for e in gold["kappa"]]
    rel_i = [abs(gI[e["cell"], e["angle"]] - e["fd"]) / max(abs(e["fd"]), fi) for e in gold["I0"]]
    report = os.environ.get("RT_ERROR_REPORT")
    if report:
        with open(report, "a") as f:
            f.write(json.dumps({"case": "adjoint_fd_64_per_cell", "precision": precision,
                                "floor": floor, "max_rel_dL_dkappa": max(rel_k),
                                "max_rel_dL_dI0": max(rel_i),
                                "max_abs_err_over_max_dL_dkappa": max(
                                    abs(gk[e["cell"]] - e["fd"]) for e in gold["kappa"]) /
                                gold["max_abs_dL_dkappa"],
                                "loss_rel": abs(L / gold["loss"] - 1)}) + "\n")
    assert max(rel_k) <= 1e-4, (max(rel_k), gold["kappa"][int(np.argmax(rel_k))])
    assert max(rel_i) <= 1e-4, (max(rel_i), gold["I0"][int(np.argmax(rel_i))])
