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


@pytest.mark.parametrize("case", list(CASES))
def test_step_io_pipeline_matches_synchronous_steps(case):
    """rt_step_io queued five times with different input rows and one output
    buffer per call (the host copies of consecutive calls overlap their
    neighbours' GPU work on the state's copy streams) against rt_set_intensity / rt_step / rt_get_intensity on a
    second state: every result and the final gas bit for bit.  A synchronous
    call after the queue (rt_get_intensity) sees the last result."""
    import torch
    prob_fn, precision = CASES[case]
    a, b = solver(prob_fn(), precision), solver(prob_fn(), precision)
    N, A = a.N, a.A
    dt = 0.5 * a.dt_limits()[1]
    rng = np.random.default_rng(11)
    K = 5
    rows = [rng.random((N, A)).astype(a.dtype) for _ in range(K)]
    pin_in = [torch.empty((N, A), dtype=a.tdtype, pin_memory=True) for _ in range(K)]
    pin_out = [torch.zeros((N, A), dtype=a.tdtype, pin_memory=True) for _ in range(K)]
    for k in range(K):
        pin_in[k].numpy()[:] = rows[k]
        a.step_io(pin_in[k], pin_out[k], dt)
    a.sync()
    for k in range(K):
        b.set_intensity(rows[k])
        b.step(dt)
        assert np.array_equal(pin_out[k].numpy(), b.get_intensity()), k
    assert np.array_equal(a.get_intensity(), pin_out[K - 1].numpy())
    ea, ma, xa = a.gas()
    eb, mb, xb = b.gas()
    assert np.array_equal(ea, eb) and np.array_equal(ma, mb) and np.array_equal(xa, xb)
    # a plain step after the queue continues from the last result
    a.step(dt)
    b.step(dt)
    assert np.array_equal(a.get_intensity(), b.get_intensity())
    a.close()
    b.close()


def test_step_io_refuses_pageable_rows():
    """Rows that are not page-locked in full take RT_ERR_ARG (the synchronous
    calls stage them instead)."""
    import torch
    prob_fn, precision = CASES["fp32_quad"]
    s = solver(prob_fn(), precision)
    N, A = s.N, s.A
    pinned = torch.zeros((N, A), dtype=s.tdtype, pin_memory=True)
    pageable = np.zeros((N, A), s.dtype)
    code = s.lib.rt_step_io(s.state, 0.0, pageable.ctypes.data, ctypes.c_void_p(pinned.data_ptr()))
    assert code == capi.RT_ERR_ARG
    code = s.lib.rt_step_io(s.state, 0.0, ctypes.c_void_p(pinned.data_ptr()), pageable.ctypes.data)
    assert code == capi.RT_ERR_ARG
    s.close()
