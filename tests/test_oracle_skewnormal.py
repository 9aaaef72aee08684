"""Pins for oracle.skewnormal (eq. 6, Section 5.1).

* n = 1: eq. (6) is Azzalini's skew-normal density with shape b / a, location xi
  and scale sqrt(a^2 + b^2) (SciPy's skewnorm), exactly (the MVN factor of a
  single variable has no QMC error).
* diagonal A and B: the product of n univariate skew-normal densities, exactly.
* n = 2 with correlated A and B: the defining integral of the model
  Z* = xi 1 + A X + B |Y| (eq. 5),
      f(z) = 2^n int_{y >= 0} phi_n(z - xi 1 - B y; A A^T) phi_n(y; I) dy,
  by adaptive quadrature, within the QMC error of the MVN factor.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import synth
from oracle import skewnormal


def test_univariate_is_azzalini_skew_normal():
    shifts = synth.lattice_shifts(3, 2, 11)
    for a, b, xi, z in ((1.0, 0.5, 0.0, 0.3), (0.7, 2.0, -0.4, -1.1), (1.3, 0.0, 0.2, 2.5), (0.5, 3.0, 0.0, -2.0)):
        lf, err = skewnormal.logpdf(np.array([z]), xi, np.array([[a]]), np.array([[b]]), shifts, 16)
        want = stats.skewnorm.logpdf(z, b / a, loc=xi, scale=math.hypot(a, b))
        assert abs(lf - want) < 1e-12 * max(1.0, abs(want)), (a, b, xi, z, lf, want)
        assert err < 1e-13 or math.isnan(err)


def test_diagonal_model_is_a_product():
    rng = np.random.default_rng(2)
    n = 5
    a = rng.uniform(0.5, 1.5, n)
    b = rng.uniform(0.1, 2.0, n)
    z = rng.normal(0.5, 1.0, n)
    xi = 0.25
    shifts = synth.lattice_shifts(2, n + 1, 12)
    lf, _ = skewnormal.logpdf(z, xi, np.diag(a), np.diag(b), shifts, 8)
    want = sum(stats.skewnorm.logpdf(z[i], b[i] / a[i], loc=xi, scale=math.hypot(a[i], b[i])) for i in range(n))
    assert abs(lf - want) < 1e-11 * abs(want)


@pytest.mark.parametrize("z", [(0.4, -0.2), (1.5, 2.0), (-1.0, 0.3)])
def test_bivariate_against_the_defining_integral(z):
    z = np.array(z)
    xi = 0.1
    A = np.array([[1.0, 0.0], [0.6, 0.8]])
    B = np.array([[0.9, 0.4], [0.4, 0.7]])
    Om1 = A @ A.T

    def integrand(y2, y1):
        y = np.array([y1, y2])
        return (stats.multivariate_normal.pdf(z - xi - B @ y, mean=np.zeros(2), cov=Om1)
                * stats.norm.pdf(y1) * stats.norm.pdf(y2))

    val, _ = integrate.dblquad(integrand, 0.0, 12.0, 0.0, 12.0, epsabs=1e-13, epsrel=1e-11)
    want = math.log(4.0 * val)
    shifts = synth.lattice_shifts(20, 3, 13)
    lf, err = skewnormal.logpdf(z, xi, A, B, shifts, 4000)
    assert abs(lf - want) <= 4 * err + 1e-7, (lf, want, err)
    # a slip in the MVN factor's limits (C = B A^-1 instead of A^-1 B) is visible
    C2 = B @ np.linalg.inv(A)
    S = np.linalg.inv(np.eye(2) + C2.T @ C2)
    bad = S @ C2.T @ np.linalg.solve(A, z - xi)
    assert np.abs(bad - skewnormal.parts(z, xi, A, B)[2]).max() > 1e-3


def test_model_matrices_follow_section_5_1():
    xy = synth.expanding_grid(4, 1.0 / 15.0, 5)
    A, B = skewnormal.model_matrices(xy, 1.0, 0.3, 0.8, 0.2)
    d = np.linalg.norm(xy[:, None, :] - xy[None, :, :], axis=2)
    assert np.allclose(A @ A.T, np.exp(-d / 0.3), atol=1e-13)
    assert np.allclose(B, 0.64 * np.exp(-d / 0.2), atol=1e-13)
    assert np.allclose(np.triu(A, 1), 0.0)
