"""Skew-normal log-density of eq. (6) (oracle; test infrastructure only).

Section 5.1: Z* = xi 1 + A X + B |Y| with X, Y independent standard normal
vectors.  Its density (eq. 6) is

    2^n phi_n(z - xi 1; A A^T + B B^T)
        * Phi_n(-inf, (I + C^T C)^-1 C^T A^-1 (z - xi 1); (I + C^T C)^-1),   C = A^-1 B.

The first factor is a normal density (plain float64 linear algebra); the second is
an MVN probability, estimated here by the dense SOV integrand of eq. (2) over the
randomly shifted Richtmyer lattice (sov.solve with a dense Cholesky factor, no
reordering).  Section 5.1's parameterisation: A the lower Cholesky factor of
sigma1^2 exp(-d / beta1) and B the covariance matrix sigma2^2 exp(-d / beta2) on
the same locations.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import cho_factor, cho_solve, cholesky, solve_triangular

from . import geometry, sov


def model_matrices(xy: np.ndarray, sigma1: float, beta1: float, sigma2: float, beta2: float):
    """(A, B) of Section 5.1: A = chol(sigma1^2 exp(-d/beta1)), B = sigma2^2 exp(-d/beta2)."""
    K1 = sigma1 ** 2 * geometry.covariance(xy, geometry.KERNEL_EXP, (beta1,), 0.0)
    K2 = sigma2 ** 2 * geometry.covariance(xy, geometry.KERNEL_EXP, (beta2,), 0.0)
    return cholesky(K1, lower=True), K2


def parts(z: np.ndarray, xi: float, A: np.ndarray, B: np.ndarray):
    """The ingredients of eq. (6): (log phi_n(z - xi 1; A A^T + B B^T), S, b*) with
    S = (I + C^T C)^-1 and b* = S C^T A^-1 (z - xi 1), C = A^-1 B."""
    n = len(z)
    r = np.asarray(z, dtype=np.float64) - xi
    Om = A @ A.T + B @ B.T
    cf = cho_factor(Om, lower=True)
    logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
    quad = float(r @ cho_solve(cf, r))
    log_phi = -0.5 * (n * math.log(2.0 * math.pi) + logdet + quad)
    C = solve_triangular(A, B, lower=True)
    M = np.eye(n) + C.T @ C
    S = np.linalg.inv(M)
    S = 0.5 * (S + S.T)
    bstar = S @ (C.T @ solve_triangular(A, r, lower=True))
    return log_phi, S, bstar


def logpdf(z: np.ndarray, xi: float, A: np.ndarray, B: np.ndarray, shifts: np.ndarray, n_points: int):
    """log of eq. (6) and the QMC error of its MVN factor: (log f, err)."""
    n = len(z)
    log_phi, S, bstar = parts(z, xi, A, B)
    L = np.linalg.cholesky(S)
    res = sov.solve(None, np.full(n, -np.inf), bstar, math.inf, shifts, n_points, L_dense=L, perm=np.arange(n))
    return n * math.log(2.0) + log_phi + res["logp"], res["err"]
