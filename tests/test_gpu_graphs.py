"""Multi-step launches through captured CUDA graphs (rt_run / rt_launch with
rt_params.plain_launches = 0) against plain launches of the same kernels:
bit-identical intensities and gas, the same launch count, and a graph that
is captured again when the arguments change (dt, buffer parity, rt_set_*)."""
import numpy as np
import pytest

from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from tests._problems import grouped, make, randomise
from tests.test_gpu_parity import solver

pytestmark = pytest.mark.gpu

G = 16  # RT_GRAPH_STEPS


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()
    capi.load()


def _pair(prob_fn, precision):
    return solver(prob_fn(), precision, plain_launches=0), solver(prob_fn(), precision, plain_launches=1)


def _same(a, b):
    assert np.array_equal(a.get_intensity(), b.get_intensity())
    for x, y in zip(a.gas(), b.gas()):
        assert np.array_equal(x, y)
    assert a.launch_count() == b.launch_count()


def _moving():
    return randomise(make(n=(7, 6, 5), order=6, cbar=10.0, c=100.0, w=(0.3, -0.1, 0.2)), seed=3)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_graph_replay_is_bit_identical(precision):
    gr, pl = _pair(_moving, precision)
    dt = 0.5 * gr.dt_limits()[1]
    for s in (gr, pl):
        s.step(dt)          # parity 1 before the multi-step call
        s.run(2 * G + 5, dt)
        s.launch(G, dt)     # queued, then synchronised by run
        s.run(G + 1, 0.5 * dt)
    _same(gr, pl)


@pytest.mark.parametrize("integrator", [0, 1], ids=["first_order", "van_leer"])
def test_graph_replay_multi_launch_steps(integrator):
    def prob():
        p = _moving()
        p.integrator = integrator
        return p
    gr, pl = _pair(prob, "fp32")
    dt = 0.5 * gr.dt_limits()[1]
    for s in (gr, pl):
        s.run(2 * G, dt)
    _same(gr, pl)


def test_graph_replay_frequency_groups():
    def prob():
        return grouped(randomise(make(n=(6, 5, 7), order=4, cbar=10.0, c=100.0), seed=4),
                       (0.4, 0.6), (0.5, 2.0), (1.0, 0.3), (0.2, 1.0), (1.0, 0.5))
    gr, pl = _pair(prob, "fp32")
    dt = 0.5 * gr.dt_limits()[1]
    for s in (gr, pl):
        s.run(G + 3, dt)
    _same(gr, pl)


def test_graph_recaptured_after_set_gas():
    base = _moving()
    gr, pl = _pair(_moving, "fp64")
    dt = 0.5 * gr.dt_limits()[1]
    for s in (gr, pl):
        s.run(G, dt)
        e, m, _ = s.gas()
        s.set_gas(base.rho, e, m, 2.0 * base.kappa_P, 0.5 * base.kappa_J, base.kappa_s)
        s.run(G, dt)
    _same(gr, pl)
