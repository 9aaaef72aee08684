"""GPU: the failure path of the tensor-core kernels' bounded waits.

Every mbarrier wait in the tcgen05 kernels gives up after a bounded number of
polls, records a code and lets the kernel free its resources and return, so a
copy or MMA that never completes becomes TLRMVN_E_TIMEOUT instead of a hang.
The self-test waits on a barrier that nothing arrives at; afterwards the CUDA
context must still run a full solve."""
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


def test_bounded_wait_gives_up_and_context_survives(tl):
    assert tl.tlrmvn_selftest_wait_timeout(1000) == tl.E_TIMEOUT
    assert b"gave up" in tl._lib.load().tlrmvn_last_error()
    assert tl.tlrmvn_selftest_wait_timeout(0) == tl.E_INVAL
    # the context is still usable: a BF16-shift solve (the path with the bounded waits)
    w = synth.small_workload(16, 64, 41, n_shifts=2, n_points=256)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 0, 2)
    lp, err, _, _ = tl.tlrmvn_prob(F, w.a, w.b, math.inf, tl.BF16_SHIFT, 2, 256, shifts=w.shifts)
    assert np.isfinite(lp) and lp < 0
