"""tlrmvn_estimate_noalloc, the estimator entry point that allocates no device memory.

It serves callers that cannot allocate (a serving loop whose device memory is
reserved up front, an application whose memory belongs to another allocator).
It must give the same estimate as tlrmvn_prob_device from the same per-sample
values, on repeated calls (its scratch is a fixed array shared by all calls),
and refuse more shifts than that array holds.  Collected last on purpose.
"""
import ctypes as C
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    from paper_2003_11183_gb300 import _lib
    return torch, tl, _lib.load()


def test_noalloc_estimate_matches_prob_on_two_calls(env):
    torch, tl, lib = env
    w = synth.small_workload(16, 64, 41, nu=7.0, n_shifts=6, n_points=300)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 0, 2)
    a = torch.tensor(w.a, dtype=torch.float64, device="cuda")
    b = torch.tensor(w.b, dtype=torch.float64, device="cuda")
    ref = torch.zeros(2, dtype=torch.float64, device="cuda")
    ref_shift = torch.zeros(w.n_shifts, dtype=torch.float64, device="cuda")
    samples = torch.zeros(w.n_shifts * w.n_points, dtype=torch.float64, device="cuda")
    tl.tlrmvn_prob_device(F, a, b, ref, nu=w.nu, precision=tl.FP32, n_shifts=w.n_shifts, n_points=w.n_points,
                          shifts=w.shifts, per_shift=ref_shift, per_sample=samples)
    torch.cuda.synchronize()
    # the first call on the device looks up the scratch array's address (set-up);
    # the calls after it must not change the device's free memory
    outs = [torch.full((2,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    pss = [torch.full((w.n_shifts,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    st = lib.tlrmvn_estimate_noalloc(samples.data_ptr(), w.n_shifts, w.n_points, outs[0].data_ptr(), None,
                                     torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.tlrmvn_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch_bytes0 = torch.cuda.memory_allocated()
    for out, ps in zip(outs, pss):
        # straight through the C ABI
        st = lib.tlrmvn_estimate_noalloc(samples.data_ptr(), w.n_shifts, w.n_points, out.data_ptr(), ps.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
        assert st == 0, lib.tlrmvn_last_error()
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.allclose(got, want, rtol=1e-12, atol=0)
        assert np.allclose(ps.cpu().numpy(), ref_shift.cpu().numpy(), rtol=1e-12, atol=0)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == torch_bytes0


def test_noalloc_rejects_too_many_shifts(env):
    torch, tl, lib = env
    from paper_2003_11183_gb300 import api
    samples = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = lib.tlrmvn_estimate_noalloc(samples.data_ptr(), api.NOALLOC_MAX_SHIFTS + 1, 1, out.data_ptr(), None, None)
    assert st == api.E_INVAL
    assert b"TLRMVN_NOALLOC_MAX_SHIFTS" in lib.tlrmvn_last_error()
