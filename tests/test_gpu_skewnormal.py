"""GPU: the skew-normal likelihood driver (eq. 6, Section 5.1) against the oracle.

* the dense parts of eq. (6) (the normal factor, the MVN problem's covariance and
  limits) equal the oracle's to rounding;
* the MVN factor through the library equals the oracle's integrand on the same
  exported factor and lattice shifts (float32 path: 1e-4 per shift);
* n = 1 reduces to Azzalini's skew-normal density;
* the batched evaluation over several parameter vectors equals one evaluation per
  vector.
"""
import math

import numpy as np
import pytest

import synth
from oracle import skewnormal as osn, sov
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
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    from paper_2003_11183_gb300 import skewnormal as sn
    return tl, sn


THETA = (0.1, 1.0, 0.3, 0.8, 0.3)


def test_dense_parts_match_the_oracle(env):
    tl, sn = env
    xy = synth.expanding_grid(10, 1.0 / 15.0, 21)
    z = sn.simulate(xy, THETA, 5)
    A, B = sn.model_matrices(sn.distances(xy), *THETA[1:])
    P = sn.parts(z, THETA[0], A, B)
    oA, oB = osn.model_matrices(xy, *THETA[1:])
    lphi, S, bstar = osn.parts(z, THETA[0], oA, oB)
    assert abs(P.log_phi - lphi) < 1e-9 * abs(lphi)
    assert np.abs(P.S.cpu().numpy() - S).max() < 1e-9
    assert np.abs(P.bstar.cpu().numpy() - bstar).max() < 1e-8 * max(1.0, np.abs(bstar).max())


def test_mvn_factor_matches_the_oracle_on_the_same_factor(env):
    # the library's factor of (I + C^T C)^-1 handed to the oracle: the float32
    # integrand's per-shift logs within 1e-4 and the log-likelihood within 1e-4
    tl, sn = env
    xy = synth.expanding_grid(16, 1.0 / 15.0, 22)
    z = sn.simulate(xy, THETA, 6)
    n = len(z)
    timings = {}
    lf, err = sn.loglik(z, xy, THETA, tile=64, tol=1e-6, n_shifts=8, n_points=500, seed=31, timings=timings)
    assert timings["dense"] > 0 and timings["mvn"] > 0
    oA, oB = osn.model_matrices(xy, *THETA[1:])
    lphi, S, bstar = osn.parts(z, THETA[0], oA, oB)
    a = np.full(n, -np.inf)
    F = tl.tlrmvn_factor_dense(S, a, bstar, 64, 1e-6, 0, tl.REORDER_BLOCK)
    OF = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F)))
    shifts = splitmix64_shifts(31, 8, n + 1)
    ref = sov.solve(OF, a, bstar, math.inf, shifts, 500)
    _, _, ps, _ = tl.tlrmvn_prob(F, a, bstar, math.inf, tl.FP32, 8, 500, seed=31, per_shift=True)
    assert np.all(np.abs(ps - ref["per_shift"]) <= 1e-4 * np.abs(ref["per_shift"]))
    want = n * math.log(2.0) + lphi + ref["logp"]
    assert abs(lf - want) <= 1e-4 * abs(want)
    # and the oracle's own dense evaluation of eq. (6) (no reordering, its own
    # shifts) estimates the same log-likelihood
    lo, eo = osn.logpdf(z, THETA[0], oA, oB, synth.lattice_shifts(8, n + 1, 32), 500)
    assert abs(lf - lo) <= 3 * math.hypot(err, eo) + 1e-6


def test_univariate_is_azzalini_skew_normal(env):
    from scipy import stats
    tl, sn = env
    xy = np.array([[0.2, 0.3]])
    for theta, z in (((0.0, 1.0, 0.3, 0.5, 0.3), 0.4), ((-0.3, 0.7, 0.3, 2.0, 0.3), -1.2)):
        lf, _ = sn.loglik(np.array([z]), xy, theta, tile=1, tol=0.0, n_shifts=2, n_points=16)
        a, b = theta[1], theta[3] ** 2  # A = chol(sigma1^2) = sigma1, B = sigma2^2 at d = 0
        want = stats.skewnorm.logpdf(z, b / a, loc=theta[0], scale=math.hypot(a, b))
        assert abs(lf - want) <= 1e-6 * max(1.0, abs(want))


def test_batch_equals_single_evaluations(env):
    tl, sn = env
    xy = synth.expanding_grid(12, 1.0 / 15.0, 23)
    z = sn.simulate(xy, THETA, 7)
    thetas = [THETA, (0.0, 1.2, 0.2, 0.5, 0.1), (0.3, 0.8, 0.5, 1.0, 0.25)]
    lb, eb = sn.loglik_batch(z, xy, thetas, tile=64, tol=1e-6, n_shifts=8, n_points=400, seed=40)
    for k, th in enumerate(thetas):
        ls, es = sn.loglik(z, xy, th, tile=64, tol=1e-6, n_shifts=8, n_points=400, seed=40 + k)
        assert abs(lb[k] - ls) <= 1e-4 * abs(ls), (k, lb[k], ls)
