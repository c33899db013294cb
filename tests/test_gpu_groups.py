"""GPU parity of frequency groups (Sec. 2.3: groups on the same angles coupled
only through the gas temperature) through the C ABI against the FP64 oracle:
RT_FP64 per intensity to a relative 1e-12, RT_FP32 in L1 of E_r to 1e-5 with
total energy conserved to 1e-6.  Two groups on S6 (96 angles, the float quad
layout) and three on S4 (72 angles, the pair layout)."""
import numpy as np
import pytest

import oracle
from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from tests._problems import grouped, make, randomise
from tests.test_gpu_parity import check_fp32, check_fp64, rel_err, solver

pytestmark = pytest.mark.gpu

FP32_ENERGY = 1e-6
CASES = [
    (6, (0.3, 0.7), (0.2, 4.0), (0.3, 2.0), (1.0, 0.1), (2.0, 0.5)),
    (4, (0.2, 0.5, 0.3), (0.3, 1.0, 3.0), (0.5, 1.0, 2.0), (2.0, 0.5, 0.0), (1.5, 1.0, 0.4)),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()
    capi.load()


def _problem(case, seed=5, w=(0.3, -0.1, 0.2)):
    order, gw, sP, sJ, sS, ig = case
    prob = randomise(make(n=(9, 7, 5), order=order, cbar=10.0, c=100.0, w=w), seed=seed)
    return grouped(prob, gw, sP, sJ, sS, ig)


@pytest.mark.parametrize("case", CASES, ids=["S6x2", "S4x3"])
@pytest.mark.parametrize("w", [None, (0.3, -0.1, 0.2)], ids=["static", "moving"])
def test_fp64_groups(case, w):
    prob = _problem(case, 5, w)
    o = oracle.Oracle(prob)
    g = solver(prob, "fp64")
    dt = o.cfl_dt()
    assert o.run(30, dt) == oracle.ORC_OK
    g.run(30, dt)
    check_fp64(o, g)


@pytest.mark.parametrize("case", CASES, ids=["S6x2", "S4x3"])
def test_fp32_groups(case):
    prob = _problem(case, 6)
    o = oracle.Oracle(prob)
    g = solver(prob, "fp32")
    t0 = g.totals()
    dt = o.cfl_dt()
    assert o.run(30, dt) == oracle.ORC_OK
    g.run(30, dt)
    check_fp32(o, g)
    t1 = g.totals()
    assert abs(t1[12] - t0[12]) < FP32_ENERGY * abs(t0[12])


def test_identical_groups_match_the_grey_kernel():
    """Two identical groups (two launches: transport, coupled source) against
    the fused grey step on the same problem."""
    base = lambda: randomise(make(n=(6, 5, 7), order=6, cbar=10.0, c=100.0, w=(0.3, 0.1, 0.0)),
                             seed=9)
    grey = solver(base(), "fp64")
    grp = solver(grouped(base(), (0.3, 0.7)), "fp64")
    dt = oracle.Oracle(base()).cfl_dt()
    grey.run(20, dt)
    grp.run(20, dt)
    Ig, Ir = grp.get_intensity(), grey.get_intensity()
    A = Ir.shape[1]
    for j in range(2):
        assert rel_err(Ig[:, j * A:(j + 1) * A], Ir) < 1e-12
    assert rel_err(grp.gas()[0], grey.gas()[0]) < 1e-12


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_groups_equilibrium(precision, tol):
    prob = grouped(make(n=(3, 4, 3), order=6, cbar=5.0, c=20.0, T=1.3, kP=2.0, kJ=2.0, kS=0.4),
                   (0.2, 0.8), scale_P=(0.1, 8.0), scale_J=(0.1, 8.0), scale_S=(3.0, 0.0))
    g = solver(prob, precision)
    I0 = g.get_intensity().astype(np.float64)
    e0, _, _ = g.gas()
    dt = 0.5 / oracle.Oracle(prob).positivity()
    g.run(3, dt)
    I = g.get_intensity().astype(np.float64)
    e, _, _ = g.gas()
    assert np.abs(I - I0).max() < tol * I0.max()
    assert np.abs(e - e0).max() < tol * e0.max()


def test_groups_refuse_what_is_grey_only():
    import torch
    prob = grouped(make(n=(4, 4, 4), order=4), (0.5, 0.5))
    g = solver(prob, "fp64")
    N, A = prob.n_cells, 2 * prob.n_angles
    t = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.RTError) as err:
        g.adjoint_step(0.01, t(N, A), t(N), t(N, 3), t(N, A), t(N), t(N, 3), t(N), t(N))
    assert err.value.code == capi.RT_ERR_STATE
    prob.integrator = capi.RT_VAN_LEER
    with pytest.raises(capi.RTError):
        solver(prob, "fp64")


@pytest.mark.parametrize("G", [4, 5], ids=["G4_tile", "G5_warp"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_groups_four_and_five(G, precision):
    """S2 with 4 groups (32 angles: the tile kernel's largest group count) and
    5 groups (40 angles: the warp-per-cell kernel)."""
    rng = np.random.default_rng(10 + G)
    gw = rng.uniform(0.5, 1.5, G)
    gw /= gw.sum()
    sP, sJ, sS, ig = (rng.uniform(0.2, 3.0, G) for _ in range(4))
    prob = grouped(randomise(make(n=(6, 5, 4), order=2, cbar=10.0, c=100.0), seed=5 + G),
                   gw, sP, sJ, sS, ig)
    o = oracle.Oracle(prob)
    g = solver(prob, precision)
    t0 = g.totals()
    dt = o.cfl_dt()
    assert o.run(30, dt) == oracle.ORC_OK
    g.run(30, dt)
    if precision == "fp64":
        check_fp64(o, g)
    else:
        check_fp32(o, g)
        assert abs(g.totals()[12] - t0[12]) < FP32_ENERGY * abs(t0[12])

