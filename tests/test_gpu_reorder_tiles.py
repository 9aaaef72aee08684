"""GPU: post-hoc within-tile reordering of a resident factor for new limits
(tlrmvn_factor_reorder_tiles) against the oracle's reorder_within_tiles on the
same factor: the same permutation (integer decisions of float64 univariate
conditioning: exact), the same factor entries to 1e-9, the float64 integrand on
it equal to the oracle's to 1e-9 per sample, a smaller QMC error than the
original order at equal N, and every precision's estimate within its tolerance."""
import math

import numpy as np
import pytest

import synth
from oracle import factor as ofactor, sov
from tests.helpers import to_oracle_factor

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


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(np.asarray(b)), 1e-300)


@pytest.mark.parametrize("side,m,ragged", [(24, 64, None), (0, 128, 700)])
def test_reorder_tiles_matches_the_oracle(tl, side, m, ragged):
    w = synth.small_workload(side, m, 90, n_shifts=10, n_points=500, tol=1e-8, ragged_n=ragged)
    F0 = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, None, None, w.m, w.tol, 0, tl.REORDER_NONE)
    OF0 = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F0)))
    rng = np.random.default_rng(3)
    b2 = rng.normal(2.5, 1.0, w.n)
    a2 = np.full(w.n, -np.inf)
    F1 = tl.tlrmvn_factor_reorder_tiles(F0, a2, b2)
    ex1 = tl.parse_export(tl.tlrmvn_factor_export(F1))
    OF1 = ofactor.reorder_within_tiles(OF0, a2, b2)
    assert np.array_equal(ex1.perm, OF1.perm)
    G1 = to_oracle_factor(ex1)
    assert max(np.abs(x - y).max() for x, y in zip(G1.B, OF1.B)) < 1e-9
    for k in OF1.U:
        if OF1.U[k].shape[1]:
            assert np.abs(G1.U[k] @ G1.V[k].T - OF1.U[k] @ OF1.V[k].T).max() < 1e-9
    lp1, err1, ps1, pm1 = tl.tlrmvn_prob(F1, a2, b2, math.inf, tl.FP64, w.n_shifts, w.n_points, shifts=w.shifts,
                                         per_shift=True, per_sample=True)
    ref = sov.solve(OF1, a2, b2, math.inf, w.shifts, w.n_points)
    assert np.all(rel(pm1, ref["per_sample"]) < 1e-9)
    lp0, err0, _, _ = tl.tlrmvn_prob(F0, a2, b2, math.inf, tl.FP64, w.n_shifts, w.n_points, shifts=w.shifts)
    assert abs(lp1 - lp0) <= 3 * math.hypot(err0, err1)
    assert err1 < err0
    for prec, tol in ((tl.FP32, 1e-4), (tl.BF16_SHIFT, 1e-2), (tl.FP16_SHIFT, 1e-2)):
        ps = tl.tlrmvn_prob(F1, a2, b2, math.inf, prec, w.n_shifts, w.n_points, shifts=w.shifts, per_shift=True)[2]
        assert np.all(rel(ps, ref["per_shift"]) < tol), prec


def test_reorder_tiles_rejects_invalid_limits(tl):
    w = synth.small_workload(8, 16, 91)
    F0 = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, None, None, w.m, w.tol, 0, tl.REORDER_NONE)
    bad = w.b.copy()
    bad[3] = np.nan
    with pytest.raises(tl.TlrmvnError) as e:
        tl.tlrmvn_factor_reorder_tiles(F0, w.a, bad)
    assert e.value.status == tl.E_INVAL
