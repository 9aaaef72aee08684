"""GPU: the convergence study's claim (Section 4, Table 3 and Fig. 3) on the
library's own factors and integrand.  For an MVN problem with the paper's
simulated limits (a = -inf, b_i ~ N(5.5, 1.25^2)) on a perturbed grid with an
exponential kernel, the geometric order, block reordering (Algorithm 4) and
iterative block reordering (Algorithm 5) estimate the same probability (every
pair within three combined standard errors), and at equal N both reorderings
give a smaller QMC error than the geometric order."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    return tl


@pytest.mark.parametrize("beta", [0.3, 0.1])
def test_reordering_lowers_the_error_at_equal_n(tl, beta):
    g = 32
    n, m = g * g, 32
    xy = synth.jittered_grid(g, 8000)
    a, b = synth.limits_normal(n, 8001, 5.5, 1.25)
    shifts = synth.lattice_shifts(10, n + 1, 8100)
    res = {}
    for reorder in (tl.REORDER_NONE, tl.REORDER_BLOCK, tl.REORDER_ITERATIVE):
        F = tl.tlrmvn_factor_kernel(xy, tl.KERNEL_EXP, (beta,), 1e-8, a, b, m, 1e-6, 0, reorder)
        lp, err, _, _ = tl.tlrmvn_prob(F, a, b, math.inf, tl.FP64, 10, 500, shifts=shifts)
        res[reorder] = (lp, err)
    for x in res.values():
        for y in res.values():
            assert abs(x[0] - y[0]) <= 3 * math.hypot(x[1], y[1])
    assert res[tl.REORDER_BLOCK][1] < res[tl.REORDER_NONE][1]
    assert res[tl.REORDER_ITERATIVE][1] < res[tl.REORDER_NONE][1]
