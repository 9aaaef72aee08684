"""Pins for oracle.special: Phi, Phi^-1, tail-safe intervals, chi quantile, truncated mean.

Pinned against 50-digit mpmath where available, closed forms, and scipy.stats.
"""
import math
import numpy as np
import pytest
from scipy import stats

from oracle import special


def test_phi_inv_round_trip():
    u = np.concatenate([np.logspace(-300, -1, 40), np.linspace(0.05, 0.95, 19), 1 - np.logspace(-1, -15, 20)])
    x = special.Phi_inv(u)
    assert np.allclose(special.Phi(x), u, rtol=1e-12, atol=0)


def test_phi_known_values():
    # textbook values of the standard normal CDF
    assert special.Phi(0.0) == 0.5
    assert abs(special.Phi(1.959963984540054) - 0.975) < 1e-15
    assert abs(special.Phi_inv(0.8413447460685429) - 1.0) < 1e-13


def _mp_log_interval(mp, a, b):
    """log(Phi(b) - Phi(a)) at the working precision; upper-half intervals through
    the complements Phi(-a) - Phi(-b), which 50 digits resolve."""
    if a > 0:
        return mp.log(mp.ncdf(-a) - (mp.mpf(0) if b == np.inf else mp.ncdf(-b)))
    fa = mp.mpf(0) if a == -np.inf else mp.ncdf(a)
    fb = mp.mpf(1) if b == np.inf else mp.ncdf(b)
    return mp.log(fb - fa)


def test_log_interval_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    cases = [(-np.inf, -30.0), (-np.inf, 0.3), (-np.inf, 9.0), (-2.0, 1.0), (1.0, 2.0), (7.0, 9.0),
             (30.0, 31.0), (-31.0, -30.0), (5.0, np.inf), (-np.inf, np.inf), (0.0, 1e-3),
             # both probabilities below the float64 range: finite in logs
             (-61.0, -60.0), (60.0, 61.0), (-41.0, -40.5), (50.0, np.inf), (-np.inf, -60.0)]
    for a, b in cases:
        want = float(_mp_log_interval(mp, a, b))
        got = float(special.log_interval(a, b))
        assert math.isfinite(want)
        assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (a, b, got, want)


def test_sov_step_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    cases = [(-np.inf, 0.5, 0.3), (-np.inf, -8.0, 0.9), (-np.inf, 6.0, 0.999), (-1.0, 2.0, 0.1),
             (3.0, 5.0, 0.5), (6.0, np.inf, 0.2), (-5.0, -4.0, 0.7),
             # deep tails: d + w (e - d) underflows in float64, y must stay finite
             (-np.inf, -60.0, 0.3), (-61.0, -60.0, 0.5), (60.0, 61.0, 0.4), (45.0, np.inf, 0.7),
             (-40.0, -39.9, 0.01)]
    for a, b, w in cases:
        wm = mp.mpf(w)
        # y solves Phi(y) = (1 - w) Phi(a) + w Phi(b); in the upper half the same
        # equation in complements, Phi(-y) = (1 - w) Phi(-a) + w Phi(-b), so that
        # 50 digits resolve it (Phi(60) = 1 - 1e-785)
        upper = a > 0
        if upper:
            target = (1 - wm) * mp.ncdf(-a) + wm * (mp.mpf(0) if b == np.inf else mp.ncdf(-b))
            g = lambda x: -mp.ncdf(-x)  # increasing in x
            target = -target
        else:
            target = (1 - wm) * (mp.mpf(0) if a == -np.inf else mp.ncdf(a)) + wm * (mp.mpf(1) if b == np.inf
                                                                                   else mp.ncdf(b))
            g = mp.ncdf
        lo, hi = mp.mpf(-80), mp.mpf(80)
        for _ in range(200):
            mid = (lo + hi) / 2
            if g(mid) < target:
                lo = mid
            else:
                hi = mid
        want_y = float((lo + hi) / 2)
        want_ld = float(_mp_log_interval(mp, a, b))
        ld, y = special.sov_step(a, b, w)
        assert math.isfinite(want_ld) and math.isfinite(float(y))
        assert abs(float(ld) - want_ld) <= 1e-12 * max(1, abs(want_ld)), (a, b, float(ld), want_ld)
        assert abs(float(y) - want_y) <= 1e-9 * max(1.0, abs(want_y)), (a, b, w, float(y), want_y)


def test_chi_inv_closed_forms():
    w = np.linspace(0.01, 0.99, 25)
    # nu = 2: S^2 ~ Exp(1/2), so chi_2^-1(w) = sqrt(-2 log(1 - w))
    assert np.allclose(special.chi_inv(2.0, w), np.sqrt(-2 * np.log1p(-w)), rtol=1e-12)
    # nu = 1: S = |Z|, so chi_1^-1(w) = Phi^-1((1 + w)/2)
    assert np.allclose(special.chi_inv(1.0, w), special.Phi_inv((1 + w) / 2), rtol=1e-12)
    # general nu: round trip through the chi CDF
    for nu in (3.0, 7.0, 10.0):
        assert np.allclose(stats.chi.cdf(special.chi_inv(nu, w), nu), w, rtol=1e-10)


def test_trunc_mean_against_scipy():
    for a, b in [(-np.inf, 0.3), (-1.0, 2.0), (2.0, np.inf), (-np.inf, -6.0), (0.5, 0.6), (-3.0, -2.5)]:
        want = stats.truncnorm.mean(a, b)
        got = float(special.trunc_mean(a, b))
        assert abs(got - want) < 1e-9 * max(1, abs(want)), (a, b, got, want)
