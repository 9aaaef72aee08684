"""GPU: the batched persistent integrand (tlrmvn_batch_*) against the oracle and
against the single-problem integrand on the same factors and shifts."""
import math

import numpy as np
import pytest

import synth
from oracle import sov
from tests.helpers import to_oracle_factor

pytestmark = pytest.mark.gpu

MASK = (1 << 64) - 1


def splitmix64_shifts(seed: int, n_shifts: int, n_coords: int) -> np.ndarray:
    """The library's seeded shifts (splitmix64 by S. Vigna): output t = mix(seed + (t+1) * golden)."""
    out = np.empty(n_shifts * n_coords, dtype=np.uint64)
    for t in range(out.size):
        z = (seed + (t + 1) * 0x9E3779B97F4A7C15) & MASK
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out[t] = z ^ (z >> 31)
    return out.reshape(n_shifts, n_coords)


@pytest.fixture(scope="module")
def tl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    return tl


def _problems(tl, sizes, m, seed0, tol=1e-8):
    out = []
    for p, n in enumerate(sizes):
        w = synth.small_workload(0, m, seed0 + p, ragged_n=n, tol=tol)
        F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 0, 2)
        out.append((w, F))
    return out


def test_batch_against_oracle(tl):
    probs = _problems(tl, [130, 300, 97, 256], 64, 50)
    nu = [math.inf, 7.0, math.inf, 3.0]
    M, N, seed = 4, 160, 1234
    lp, err = tl.tlrmvn_prob_batch([F for _, F in probs], [w.a for w, _ in probs], [w.b for w, _ in probs], nu, M, N,
                                   seed=seed)
    for p, (w, F) in enumerate(probs):
        OF = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F)))
        D = splitmix64_shifts(seed + p, M, w.n + 1)
        ref = sov.solve(OF, w.a, w.b, nu[p], D, N)
        assert abs(lp[p] - ref["logp"]) <= 1e-4 * abs(ref["logp"]), (p, lp[p], ref["logp"])
        assert abs(err[p] - ref["err"]) <= 1e-2 * ref["err"] + 1e-6


def test_batch_matches_single_problem_path(tl):
    probs = _problems(tl, [700, 1024, 333], 128, 60, tol=1e-6)
    M, N, seed = 3, 1000, 99
    plan = tl.BatchPlan([F for _, F in probs], math.inf, M, N, seed=seed)
    lp, err = plan.run([w.a for w, _ in probs], [w.b for w, _ in probs])
    for p, (w, F) in enumerate(probs):
        l1, e1, _, _ = tl.tlrmvn_prob(F, w.a, w.b, math.inf, tl.FP32, M, N, seed=seed + p)
        assert abs(lp[p] - l1) <= 1e-4 * abs(l1)
    plan.close()


def test_batch_plan_replays_with_new_limits(tl):
    probs = _problems(tl, [200, 150], 64, 70)
    plan = tl.BatchPlan([F for _, F in probs], [math.inf, 5.0], 2, 256, seed=5)
    a1 = [w.a for w, _ in probs]
    b1 = [w.b for w, _ in probs]
    b2 = [w.b + 0.5 for w, _ in probs]
    r1 = plan.run(a1, b1)
    r2 = plan.run(a1, b2)
    r3 = plan.run(a1, b1)
    assert np.array_equal(r1[0], r3[0]) and np.array_equal(r1[1], r3[1])
    assert np.all(r2[0] > r1[0])  # wider limits, larger probability
    with pytest.raises(tl.TlrmvnError) as e:
        plan.run(a1, [np.full_like(b, np.nan) for b in b1])
    assert e.value.status == tl.E_INVAL
    r4 = plan.run(a1, b1)  # the plan stays usable after a rejected call
    assert np.array_equal(r1[0], r4[0])
    plan.close()


# ---- the tensor-core batched kernel (TLRMVN_BF16_SHIFT) ----------------------------------

def test_batch_bf16_against_oracle(tl):
    # tiles of 64 and 128 (one and two 64-variable sub-tiles: the split-bf16 coupling),
    # ragged last tiles, MVN and MVT: every problem's estimate within the BF16-shift
    # tolerance of the oracle's on the same factor and shifts (1e-2 relative and 3 SE)
    probs = _problems(tl, [130, 300, 97], 64, 80) + _problems(tl, [700, 333], 128, 85, tol=1e-6)
    nu = [math.inf, 7.0, math.inf, 3.0, math.inf]
    M, N, seed = 4, 300, 4321
    lp, err = tl.tlrmvn_prob_batch([F for _, F in probs], [w.a for w, _ in probs], [w.b for w, _ in probs], nu, M, N,
                                   seed=seed, precision=tl.BF16_SHIFT)
    for p, (w, F) in enumerate(probs):
        OF = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F)))
        D = splitmix64_shifts(seed + p, M, w.n + 1)
        ref = sov.solve(OF, w.a, w.b, nu[p], D, N)
        assert abs(lp[p] - ref["logp"]) <= 1e-2 * abs(ref["logp"]), (p, lp[p], ref["logp"])
        assert abs(lp[p] - ref["logp"]) <= 3 * math.hypot(err[p], ref["err"]) + 1e-3 * abs(ref["logp"]), p


def test_batch_bf16_matches_single_problem_bf16_path(tl):
    # the same whole-tile sweep per tile, only the samples' placement differs: the
    # batched estimate equals the single-problem BF16-shift path's on the same shifts
    probs = _problems(tl, [700, 1024, 333, 2000], 128, 90, tol=1e-6)
    nu = [math.inf, 7.0, math.inf, math.inf]
    M, N, seed = 3, 1000, 17
    plan = tl.BatchPlan([F for _, F in probs], nu, M, N, seed=seed, precision=tl.BF16_SHIFT)
    lp, err = plan.run([w.a for w, _ in probs], [w.b for w, _ in probs])
    for p, (w, F) in enumerate(probs):
        l1, e1, _, _ = tl.tlrmvn_prob(F, w.a, w.b, nu[p], tl.BF16_SHIFT, M, N, seed=seed + p)
        assert abs(lp[p] - l1) <= 1e-6 * abs(l1), (p, lp[p], l1)
        assert abs(err[p] - e1) <= 1e-4 * e1 + 1e-9
    # replay with new limits, then the old ones again: identical results
    lp2, _ = plan.run([w.a for w, _ in probs], [w.b + 0.3 for w, _ in probs])
    assert np.all(lp2 > lp)
    lp3, err3 = plan.run([w.a for w, _ in probs], [w.b for w, _ in probs])
    assert np.array_equal(lp, lp3) and np.array_equal(err, err3)
    # the tuned grid gives the same results
    got = plan.tune([w.a for w, _ in probs], [w.b for w, _ in probs], None, True)
    assert got["ctas_per_sm"] >= 1
    lp4, _ = plan.run([w.a for w, _ in probs], [w.b for w, _ in probs])
    assert np.allclose(lp4, lp, rtol=1e-6, atol=0)
    plan.close()


def test_batch_rejects_other_precisions(tl):
    probs = _problems(tl, [100], 64, 95)
    with pytest.raises(tl.TlrmvnError) as e:
        tl.BatchPlan([F for _, F in probs], math.inf, 2, 64, precision=tl.FP64)
    assert e.value.status == tl.E_NOTSUP
