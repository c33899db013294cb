"""rt_totals_noalloc: conserved totals with no device allocation.

The entry point serves callers that cannot call cudaMalloc (code running
where the allocator is off limits, or whose device memory is owned by
another allocator): it keeps its partial sums in a static device array of
the library instead of a buffer rt_create allocated.  This checks it
against rt_totals, through the C ABI, on two calls in a row.  The file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2002_08377_gb300 import build as rtbuild
from paper_2002_08377_gb300 import capi
from tests._problems import make, randomise

pytestmark = pytest.mark.gpu


def _pair(lib, g):
    ref = np.empty(16)
    assert lib.rt_totals(g.state, ref.ctypes.data) == capi.RT_OK
    got = np.empty(16)
    code = lib.rt_totals_noalloc(g.state, got.ctypes.data)
    assert code == capi.RT_OK, lib.rt_last_error(g.state)
    return ref, got


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_totals_noalloc_matches_totals(precision):
    """Up to 131,072 cells the blocks are rt_totals' own: bit-identical."""
    rtbuild.build()
    lib = capi.load()
    from paper_2002_08377_gb300.solver import RTSolver
    prob = randomise(make(n=(9, 7, 5), order=6, cbar=10.0, c=100.0), seed=21)
    g = RTSolver.from_problem(prob, precision)
    for _ in range(2):
        g.run(3)
        ref, got = _pair(lib, g)
        assert np.array_equal(got, ref)
    g.close()


def test_totals_noalloc_large_then_small_state():
    """A state above 2048 x 64 cells (60^3: larger blocks, the same totals to
    rounding), then a smaller one whose call reads only what it wrote
    (bit-identical to rt_totals), two calls each."""
    rtbuild.build()
    lib = capi.load()
    from paper_2002_08377_gb300.inputs import shadows
    from paper_2002_08377_gb300.solver import RTSolver
    big = RTSolver.from_problem(shadows(n=60, steps=2), "fp32")
    assert big.N > 2048 * 64
    for _ in range(2):
        big.run(2)
        ref, got = _pair(lib, big)
        scale = np.abs(ref).max()
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-13 * scale)
    big.close()
    small = RTSolver.from_problem(randomise(make(n=(5, 6, 7), order=4), seed=3), "fp64")
    for _ in range(2):
        small.run(2)
        ref, got = _pair(lib, small)
        assert np.array_equal(got, ref)
    small.close()
