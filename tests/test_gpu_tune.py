"""GPU: the autotuners (tlrmvn_autotune, tlrmvn_batch_tune).  A tuned launch
choice changes how the integrand is launched, never what it computes: every
candidate still matches the oracle on the same factor, lattice and shifts, a
cached choice is read back without timing, and a tuned batch plan gives its
untuned results bit for bit."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import sov
from tests.helpers import to_oracle_factor, oracle_factor, export_bytes

pytestmark = pytest.mark.gpu

TOL = {"FP64": 1e-9, "FP32": 1e-4, "BF16_SHIFT": 1e-2}


@pytest.fixture(scope="module")
def tl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    return tl


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(np.asarray(b)), 1e-300)


@pytest.mark.parametrize("precision", ["FP64", "FP32", "BF16_SHIFT"])
def test_tuned_choice_matches_the_oracle(tl, tmp_path, precision):
    # tiles of 256: four 64-variable sub-tiles (two of 128), so the sub-tile and
    # block-size candidates all differ; Student-t, ragged last tile
    w = synth.small_workload(0, 256, 61, nu=7.0, n_shifts=4, n_points=600, ragged_n=700)
    OF, _ = oracle_factor(w)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    prec = getattr(tl, precision)
    cache = str(tmp_path / "tune.txt")
    kw = dict(n_shifts=w.n_shifts, n_points=w.n_points, shifts=w.shifts)
    got = tl.tlrmvn_autotune(F, w.a, w.b, w.nu, prec, cache_path=cache, **kw)
    assert got["candidates"] >= 2 and got["ms"] > 0
    assert tl.tlrmvn_get_tuning(F, prec)["sub"] == got["sub"]
    ref = sov.solve(OF, w.a, w.b, w.nu, w.shifts, w.n_points)
    lp, err, ps, pm = tl.tlrmvn_prob(F, w.a, w.b, w.nu, prec, per_shift=True, per_sample=True, **kw)
    assert np.all(rel(ps, ref["per_shift"]) < TOL[precision])
    # the cache gives the same choice back without timing
    F2 = tl.tlrmvn_factor_import(export_bytes(OF))
    again = tl.tlrmvn_autotune(F2, w.a, w.b, w.nu, prec, cache_path=cache, **kw)
    assert again["candidates"] == 0 and again["ms"] == -1.0
    assert {k: again[k] for k in ("sub", "threads", "chunk", "tc_ctas", "spt")} == \
        {k: got[k] for k in ("sub", "threads", "chunk", "tc_ctas", "spt")}
    assert os.path.getsize(cache) > 0


def test_every_float32_candidate_matches_the_oracle(tl):
    w = synth.small_workload(0, 256, 62, n_shifts=3, n_points=500, ragged_n=650)
    OF, _ = oracle_factor(w)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    ref = sov.solve(OF, w.a, w.b, w.nu, w.shifts, w.n_points)
    kw = dict(n_shifts=w.n_shifts, n_points=w.n_points, shifts=w.shifts, per_shift=True, per_sample=True)
    for sub in (64, 128):
        for threads in (0, 64, 128, 256):
            for chunk in (0, 512):
                tl.tlrmvn_set_tuning(F, tl.FP32, sub=sub, threads=threads, chunk=chunk)
                lp, err, ps, pm = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP32, **kw)
                assert np.all(rel(ps, ref["per_shift"]) < 1e-4), (sub, threads, chunk)
                assert np.all(rel(pm, ref["per_sample"]) < 1e-4), (sub, threads, chunk)
    with pytest.raises(tl.TlrmvnError) as e:
        tl.tlrmvn_set_tuning(F, tl.FP32, sub=96)
    assert e.value.status == tl.E_INVAL


def test_bf16_candidates_give_identical_samples(tl):
    # the whole-tile sweep's launch choices (CTAs per SM, samples per pass) do not
    # change a single sample: every product and sum runs in the same order
    w = synth.small_workload(0, 128, 63, nu=3.0, n_shifts=4, n_points=700, ragged_n=500)
    OF, _ = oracle_factor(w)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    kw = dict(n_shifts=w.n_shifts, n_points=w.n_points, shifts=w.shifts, per_sample=True)
    base = None
    for ctas, spt in ((6, 1), (4, 1), (2, 1), (4, 2), (2, 2)):
        for chunk in (0, 768):
            tl.tlrmvn_set_tuning(F, tl.BF16_SHIFT, tc_ctas=ctas, chunk=chunk, spt=spt)
            pm = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.BF16_SHIFT, **kw)[3]
            if base is None:
                base = pm
            assert np.array_equal(pm, base), (ctas, spt, chunk)
    ref = sov.solve(OF, w.a, w.b, w.nu, w.shifts, w.n_points)
    assert np.all(rel(base, ref["per_sample"]) < 1e-2)
    # the FP16-shift path: two samples per thread give the same samples as one
    tl.tlrmvn_set_tuning(F, tl.FP16_SHIFT, spt=1)
    p1 = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP16_SHIFT, **kw)[3]
    tl.tlrmvn_set_tuning(F, tl.FP16_SHIFT, tc_ctas=4, spt=2)
    p2 = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP16_SHIFT, **kw)[3]
    assert np.array_equal(p1, p2)
    assert np.all(rel(p2, ref["per_sample"]) < 1e-2)


def test_batch_tune_keeps_results(tl, tmp_path):
    sizes = [300, 130, 512, 97, 256, 700]
    probs = []
    for p, n in enumerate(sizes):
        w = synth.small_workload(0, 64 if p % 2 else 128, 70 + p, ragged_n=n, tol=1e-6)
        probs.append((w, tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 0, 1)))
    nu = [math.inf, 7.0] * 3
    plan = tl.BatchPlan([F for _, F in probs], nu, 4, 300, seed=99)
    a, b = [w.a for w, _ in probs], [w.b for w, _ in probs]
    lp0, er0 = plan.run(a, b)
    cache = str(tmp_path / "batch_tune.txt")
    choice = plan.tune(a, b, cache_path=cache)
    assert choice["ctas_per_sm"] >= 1 and choice["ms"] > 0
    lp1, er1 = plan.run(a, b)
    assert np.array_equal(lp0, lp1) and np.array_equal(er0, er1)
    again = plan.tune(a, b, cache_path=cache)
    assert again["ctas_per_sm"] == choice["ctas_per_sm"] and again["ms"] == -1.0
    plan.close()
