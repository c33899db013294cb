"""Intensity I/O through the C ABI with host buffers: page-locked host rows
(read and written by one permute pass over the host link) against pageable
rows (staged copy, then the permute) and device rows — bit-identical, in
the float quad layout, the pair layout (FP64) and with frequency groups."""
import ctypes

import numpy as np
import pytest

from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from tests._problems import grouped, make, randomise
from tests.test_gpu_parity import solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()
    capi.load()


CASES = {
    "fp32_quad": (lambda: randomise(make(n=(7, 6, 5), order=8, cbar=10.0, c=100.0), seed=2), "fp32"),
    "fp64_pairs": (lambda: randomise(make(n=(7, 6, 5), order=6, cbar=10.0, c=100.0), seed=2), "fp64"),
    "fp32_groups": (lambda: grouped(randomise(make(n=(6, 5, 7), order=4, cbar=10.0, c=100.0), seed=4),
                                    (0.4, 0.6), (0.5, 2.0), (1.0, 0.3), (0.2, 1.0), (1.0, 0.5)), "fp32"),
}


@pytest.mark.parametrize("case", list(CASES))
def test_pinned_host_io_is_bit_identical(case):
    import torch
    prob_fn, precision = CASES[case]
    s = solver(prob_fn(), precision)
    N, A = s.N, s.A
    I = np.random.default_rng(5).random((N, A)).astype(s.dtype)
    pin_in = torch.empty((N, A), dtype=s.tdtype, pin_memory=True)
    pin_in.numpy()[:] = I
    pin_out = torch.zeros((N, A), dtype=s.tdtype, pin_memory=True)
    lib, st = s.lib, s.state
    p_in, p_out = ctypes.c_void_p(pin_in.data_ptr()), ctypes.c_void_p(pin_out.data_ptr())
    # pinned in, pageable and pinned and device out
    s._check(lib.rt_set_intensity(st, p_in, 0))
    assert np.array_equal(s.get_intensity(), I)
    s._check(lib.rt_get_intensity(st, p_out, 0))
    assert np.array_equal(pin_out.numpy(), I)
    assert np.array_equal(s.get_intensity(device=True).cpu().numpy(), I)
    # one step from each loading path gives the same state
    dt = 0.5 * s.dt_limits()[1]
    s.step(dt)
    after_pinned = s.get_intensity()
    s2 = solver(prob_fn(), precision)
    s2.set_intensity(I)
    s2.step(dt)
    assert np.array_equal(s2.get_intensity(), after_pinned)
    s2._check(s2.lib.rt_get_intensity(s2.state, p_out, 0))
    assert np.array_equal(pin_out.numpy(), after_pinned)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_set_gas_energy_restores_a_checkpoint(precision):
    """rt_set_gas_energy with device tensors (and with host arrays) restores
    (e, m) saved after a few steps: the steps that follow are bit-identical
    to those after the save."""
    import torch
    from paper_2002_08377_gb300.solver import RTSolver
    prob = randomise(make(n=(6, 5, 7), order=6, cbar=10.0, c=30.0), seed=4, kinds=False)
    g = RTSolver.from_problem(prob, precision)
    g.run(3)
    I = g.get_intensity(device=True).clone()
    e, m = g.gas_device()
    e, m = e.clone(), m.clone()
    g.run(4)
    ref_I, (ref_e, ref_m, _) = g.get_intensity(), g.gas()
    for src in ((e, m), (e.cpu().numpy(), m.cpu().numpy())):
        g.set_gas_energy(*src)
        g.set_intensity(I)
        g.run(4)
        assert np.array_equal(g.get_intensity(), ref_I)
        e2, m2, _ = g.gas()
        assert np.array_equal(e2, ref_e) and np.array_equal(m2, ref_m)
    g.close()
