"""GPU: the serving loop (tlrmvn_server_*): continuous admission, overlap on the
device, and results that are the same alone and in the mix."""
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
    ws, fs = [], []
    for seed, (side, m) in enumerate([(24, 64), (32, 128), (40, 128)]):
        w = synth.small_workload(side, m, 80 + seed, tol=1e-6)
        fs.append(tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 0, 2))
        ws.append(w)
    return tl, ws, fs


def _req(w, k, rng):
    b = rng.uniform(0.0, 1.0, w.n)
    return np.full(w.n, -np.inf), b, [math.inf, 7.0, 3.0][k % 3], [1, 2][k % 2]


def test_same_alone_and_in_the_mix(env):
    tl, ws, fs = env
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(12):
        f = k % 3
        a, b, nu, prec = _req(ws[f], k, rng)
        reqs.append((f, a, b, nu, prec))
    kw = dict(n_shifts=4, n_points=2000, seed=11)
    # alone: one request at a time
    alone = []
    srv = tl.Server(fs, lanes=4, memory_budget=8 << 30)
    for f, a, b, nu, prec in reqs:
        rid = srv.submit(f, a, b, nu, prec, **kw)
        alone.append(srv.wait(rid)[:2])
    # in the mix: all submitted at once
    ids = [srv.submit(f, a, b, nu, prec, **kw) for f, a, b, nu, prec in reqs]
    mixed = [srv.wait(i)[:2] for i in ids]
    st = srv.stats()
    srv.close()
    for (l1, e1), (l2, e2) in zip(alone, mixed):
        assert l1 == l2 and (e1 == e2 or (math.isnan(e1) and math.isnan(e2)))
    assert st["completed"] == 24
    assert st["peak_in_flight"] > 1 and st["overlapped"] > 0
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # and the same as the plain entry point
    f, a, b, nu, prec = reqs[0]
    lp, err, _, _ = tl.tlrmvn_prob(fs[f], a, b, nu, prec, **kw)
    assert lp == alone[0][0] and err == alone[0][1]


def test_admission_by_memory_budget(env):
    tl, ws, fs = env
    rng = np.random.default_rng(1)
    a, b, nu, prec = _req(ws[2], 0, rng)
    # a budget of 1.5 requests admits exactly one at a time
    kw = dict(n_shifts=4, n_points=4000, seed=3, sample_chunk=2048)
    one = tl.tlrmvn_prob_scratch_bytes(fs[2], tl.FP32, 4, 4000, sample_chunk=2048)
    budget = int(1.5 * one)
    srv = tl.Server(fs, lanes=4, memory_budget=budget)
    ids = [srv.submit(2, a, b, nu, tl.FP32, **kw) for _ in range(6)]
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    assert st["peak_in_flight"] == 1 and st["peak_bytes"] == one
    assert all(r[0] == res[0][0] for r in res)
    # a request that can never fit the budget: admission refused
    with pytest.raises(tl.TlrmvnError) as e:
        srv.submit(2, a, b, nu, tl.FP32, n_shifts=20, n_points=200000)
    assert e.value.status == tl.E_BUSY
    with pytest.raises(tl.TlrmvnError) as e:
        srv.submit(7, a, b, nu, tl.FP32, **kw)
    assert e.value.status == tl.E_INVAL
    srv.close()


def test_served_results_match_the_oracle(env):
    # one request per (precision, nu) class, served in a mix, against the oracle on
    # the same factor, lattice and shifts: FP32 within 1e-4 relative of the oracle's
    # log-probability, BF16-shift within 1e-2 relative and 3 QMC standard errors
    from oracle import sov
    from tests.helpers import to_oracle_factor
    tl, ws, fs = env
    rng = np.random.default_rng(5)
    M, N = 4, 500
    classes = [(prec, nu) for prec in (tl.FP32, tl.BF16_SHIFT) for nu in (math.inf, 7.0, 3.0)]
    srv = tl.Server(fs, lanes=4, memory_budget=8 << 30)
    reqs = []
    for k, (prec, nu) in enumerate(classes):
        f = (k + 1) % 3          # tiles of 64 and of 128 (the whole-tile sweep on the BF16 path)
        w = ws[f]
        b = rng.uniform(0.0, 1.0, w.n)
        shifts = synth.lattice_shifts(M, w.n + 1, 900 + k)
        rid = srv.submit(f, np.full(w.n, -np.inf), b, nu, prec, n_shifts=M, n_points=N, shifts=shifts)
        reqs.append((rid, f, b, nu, prec, shifts))
    got = [srv.wait(r[0]) for r in reqs]
    srv.close()
    OFs = {}
    for (rid, f, b, nu, prec, shifts), (lp, err, _) in zip(reqs, got):
        if f not in OFs:
            OFs[f] = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(fs[f])))
        ref = sov.solve(OFs[f], np.full(ws[f].n, -np.inf), b, nu, shifts, N)
        if prec == tl.FP32:
            assert abs(lp - ref["logp"]) <= 1e-4 * abs(ref["logp"]), (prec, nu, lp, ref["logp"])
        else:
            assert abs(lp - ref["logp"]) <= 1e-2 * abs(ref["logp"]), (prec, nu, lp, ref["logp"])
            assert abs(lp - ref["logp"]) <= 3 * max(err, ref["err"])
