"""Univariate special functions of the SOV integrand (oracle; test infrastructure only).

Section 2.1 of the paper: the SOV integrand needs only the standard normal CDF
Phi and its quantile Phi^-1 (the paper takes them from Intel MKL; here scipy).
Section 2.2, eq. (4b) and Algorithm 3: the Student-t problem scales the limits
by chi_nu^-1(w0)/sqrt(nu), where chi_nu^-1 is the quantile of the chi
distribution with nu degrees of freedom.
"""
from __future__ import annotations

import math
import numpy as np
from scipy import special as sp

_LOG_SQRT_2PI = 0.5 * math.log(2.0 * math.pi)


def Phi(x):
    """Standard normal CDF (scipy.special.ndtr)."""
    return sp.ndtr(x)


def log_Phi(x):
    """log Phi(x), accurate in the lower tail (scipy.special.log_ndtr)."""
    return sp.log_ndtr(x)


def Phi_inv(u):
    """Standard normal quantile (scipy.special.ndtri)."""
    return sp.ndtri(u)


def log_phi(x):
    """log of the standard normal density."""
    x = np.asarray(x, dtype=np.float64)
    return -0.5 * x * x - _LOG_SQRT_2PI


def chi_inv(nu: float, w0):
    """Quantile of the chi distribution with nu degrees of freedom.

    S ~ chi_nu  <=>  S^2/2 ~ Gamma(nu/2, 1), so chi_nu^-1(w) = sqrt(2 P^-1(nu/2, w))
    with P the regularised lower incomplete gamma function (scipy.special.gammaincinv).
    """
    return np.sqrt(2.0 * sp.gammaincinv(0.5 * nu, w0))


def log_interval(at, bt):
    """log(Phi(bt) - Phi(at)) for at <= bt, elementwise, without cancellation or underflow.

    Lower half (bt <= 0): log Phi(bt) + log(-expm1(log Phi(at) - log Phi(bt))),
    which stays finite when both probabilities underflow.  Upper half (at > 0):
    the same with the upper-tail complements Phi(-at) - Phi(-bt).  Intervals
    that straddle 0 take the plain difference (it is at least Phi(bt) - 1/2).
    """
    at = np.asarray(at, dtype=np.float64)
    bt = np.asarray(bt, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        la, lb = log_Phi(at), log_Phi(bt)
        lca, lcb = log_Phi(-at), log_Phi(-bt)
        low = lb + np.log(-np.expm1(la - lb))
        up = lca + np.log(-np.expm1(lcb - lca))
        mid = np.log(Phi(bt) - Phi(at))
        out = np.where(bt <= 0, low, np.where(at > 0, up, mid))
        out = np.where(np.isneginf(at), lb, out)
        out = np.where(np.isposinf(bt) & (at > 0), lca, out)
    return out


def sov_step(at, bt, w):
    """One variable of eq. (2): returns (log(e - d), y) for standardised limits.

    d = Phi(at), e = Phi(bt), y = Phi^-1(d + w (e - d)).  The quantile is taken
    from the log of its argument, d + w (e - d) = (1 - w) d + w e, so that it
    stays finite in the tails where the argument underflows
    (scipy.special.ndtri_exp).  In the upper half (at > 0) the same y is
    -Phi^-1((1 - w) Phi(-at) + w Phi(-bt)) by symmetry.
    """
    at = np.asarray(at, dtype=np.float64)
    bt = np.asarray(bt, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        l1w, lw = np.log1p(-w), np.log(w)
        upper = at > 0
        lu = np.logaddexp(l1w + log_Phi(at), lw + log_Phi(bt))
        luc = np.logaddexp(l1w + log_Phi(-at), lw + log_Phi(-bt))
        y = np.where(upper, -sp.ndtri_exp(luc), sp.ndtri_exp(lu))
    return log_interval(at, bt), y


def trunc_mean(at, bt):
    """Mean of a standard normal truncated to (at, bt): (phi(at) - phi(bt)) / (Phi(bt) - Phi(at)).

    Used by univariate conditioning (the truncated expectations of Algorithm 5).
    Written as exp(log phi - log(Phi(bt) - Phi(at))) for each density term so the
    ratio stays finite far in the tails.
    """
    at = np.asarray(at, dtype=np.float64)
    bt = np.asarray(bt, dtype=np.float64)
    ld = log_interval(at, bt)
    with np.errstate(over="ignore", invalid="ignore"):
        ta = np.where(np.isfinite(at), np.exp(log_phi(np.where(np.isfinite(at), at, 0.0)) - ld), 0.0)
        tb = np.where(np.isfinite(bt), np.exp(log_phi(np.where(np.isfinite(bt), bt, 0.0)) - ld), 0.0)
    return ta - tb
