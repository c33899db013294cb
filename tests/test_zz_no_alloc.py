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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_totals_noalloc_matches_totals(precision):
    rtbuild.build()
    lib = capi.load()
    from paper_2002_08377_gb300.solver import RTSolver
    prob = randomise(make(n=(9, 7, 5), order=6, cbar=10.0, c=100.0), seed=21)
    g = RTSolver.from_problem(prob, precision)
    for _ in range(2):
        g.run(3)
        ref = np.empty(16)
        assert lib.rt_totals(g.state, ref.ctypes.data) == capi.RT_OK
        got = np.empty(16)
        code = lib.rt_totals_noalloc(g.state, got.ctypes.data)
        assert code == capi.RT_OK, lib.rt_last_error(g.state)
        scale = np.abs(ref).max()
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * scale)
    g.close()
