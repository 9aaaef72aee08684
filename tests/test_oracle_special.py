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


def test_log_interval_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    cases = [(-np.inf, -30.0), (-np.inf, 0.3), (-np.inf, 9.0), (-2.0, 1.0), (1.0, 2.0), (7.0, 9.0),
             (30.0, 31.0), (-31.0, -30.0), (5.0, np.inf), (-np.inf, np.inf), (0.0, 1e-3)]
    for a, b in cases:
        fa = mp.mpf(0) if a == -np.inf else mp.ncdf(a)
        fb = mp.mpf(1) if b == np.inf else mp.ncdf(b)
        want = float(mp.log(fb - fa))
        got = float(special.log_interval(a, b))
        assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (a, b, got, want)


def test_sov_step_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    cases = [(-np.inf, 0.5, 0.3), (-np.inf, -8.0, 0.9), (-np.inf, 6.0, 0.999), (-1.0, 2.0, 0.1),
             (3.0, 5.0, 0.5), (6.0, np.inf, 0.2), (-5.0, -4.0, 0.7)]
    for a, b, w in cases:
        fa = mp.mpf(0) if a == -np.inf else mp.ncdf(a)
        fb = mp.mpf(1) if b == np.inf else mp.ncdf(b)
        u = fa + mp.mpf(w) * (fb - fa)
        # Phi^-1(u) by bisection at 50 digits
        lo, hi = mp.mpf(-40), mp.mpf(40)
        for _ in range(200):
            mid = (lo + hi) / 2
            if mp.ncdf(mid) < u:
                lo = mid
            else:
                hi = mid
        want_y = float((lo + hi) / 2)
        ld, y = special.sov_step(a, b, w)
        assert abs(float(ld) - float(mp.log(fb - fa))) <= 1e-12 * max(1, abs(float(mp.log(fb - fa))))
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
