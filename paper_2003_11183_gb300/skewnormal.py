"""Skew-normal likelihood of eq. (6) on the GPU, the application of Section 5.

Z* = xi 1 + A X + B |Y| (eq. 5) has the density

    2^n phi_n(z - xi 1; A A^T + B B^T)
        * Phi_n(-inf, (I + C^T C)^-1 C^T A^-1 (z - xi 1); (I + C^T C)^-1),   C = A^-1 B,

with Section 5.1's parameterisation theta = (xi, sigma1, beta1, sigma2, beta2): A
the lower Cholesky factor of sigma1^2 exp(-d / beta1) and B the covariance matrix
sigma2^2 exp(-d / beta2) on the data's locations.  The dense O(n^3) algebra of the
normal factor and of the MVN problem's covariance and limits (Section 5.1 names it
as the dominant cost) runs on the GPU in float64 through torch.linalg (cuSOLVER /
cuBLAS); the MVN probability, the factor the paper's method is for, is the
library's: the block-reordered TLR Cholesky factor of (I + C^T C)^-1
(tlrmvn_factor_dense) and the TLR quasi-Monte Carlo integrand (tlrmvn_prob), or,
for many parameter vectors at once as a likelihood optimiser needs, one batched
persistent launch over all their factors (tlrmvn_prob_batch).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import api


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the skew-normal likelihood needs a CUDA device")
    return torch


def distances(xy, device="cuda"):
    """Pairwise distances of the locations (float64, on the device)."""
    torch = _torch()
    p = torch.as_tensor(np.asarray(xy, dtype=np.float64), device=device)
    # (the difference form: the matrix-product form leaves ~1e-9 instead of 0 on the diagonal)
    return torch.cdist(p, p, compute_mode="donot_use_mm_for_euclid_dist")


def model_matrices(D, sigma1: float, beta1: float, sigma2: float, beta2: float):
    """(A, B) of Section 5.1 from the distance matrix D (device, float64)."""
    torch = _torch()
    K1 = sigma1 ** 2 * torch.exp(-D / beta1)
    B = sigma2 ** 2 * torch.exp(-D / beta2)
    return torch.linalg.cholesky(K1), B


@dataclass
class Parts:
    log_phi: float      # log phi_n(z - xi 1; A A^T + B B^T)
    S: object           # (I + C^T C)^-1, device float64
    bstar: object       # S C^T A^-1 (z - xi 1), device float64


def parts(z, xi: float, A, B) -> Parts:
    """The normal factor of eq. (6) and the MVN problem of its second factor."""
    torch = _torch()
    n = A.shape[0]
    r = torch.as_tensor(np.asarray(z, dtype=np.float64), device=A.device) - xi
    Om = A @ A.T + B @ B.T
    Lo = torch.linalg.cholesky(Om)
    logdet = 2.0 * torch.log(torch.diagonal(Lo)).sum()
    u = torch.linalg.solve_triangular(Lo, r[:, None], upper=False)
    log_phi = -0.5 * (n * math.log(2.0 * math.pi) + logdet + (u * u).sum())
    C = torch.linalg.solve_triangular(A, B, upper=False)
    M = torch.eye(n, dtype=torch.float64, device=A.device) + C.T @ C
    S = torch.cholesky_inverse(torch.linalg.cholesky(M))
    S = 0.5 * (S + S.T)
    bstar = S @ (C.T @ torch.linalg.solve_triangular(A, r[:, None], upper=False))[:, 0]
    return Parts(float(log_phi), S, bstar)


def loglik(z, xy, theta, tile: int = 128, tol: float = 1e-5, n_shifts: int = 10, n_points: int = 1000,
           seed: int = 0, precision: int = api.FP32, reorder: int = api.REORDER_BLOCK, D=None, timings=None):
    """log f(z; theta) of eq. (6) with its QMC error (the error of the MVN factor's
    log, i.e. its relative error); theta = (xi, sigma1, beta1, sigma2, beta2).
    `timings`, if a dict, receives the seconds of the dense algebra and of the MVN
    probability (factor + integrand)."""
    torch = _torch()
    xi, s1, b1, s2, b2 = theta
    n = len(z)
    t0 = time.perf_counter()
    D = distances(xy) if D is None else D
    A, B = model_matrices(D, s1, b1, s2, b2)
    P = parts(z, xi, A, B)
    S = P.S.cpu().numpy()
    bstar = P.bstar.cpu().numpy()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    a = np.full(n, -np.inf)
    F = api.tlrmvn_factor_dense(S, a, bstar, tile, tol, 0, reorder)
    lp, err, _, _ = api.tlrmvn_prob(F, a, bstar, math.inf, precision, n_shifts, n_points, seed=seed)
    F.close()
    t2 = time.perf_counter()
    if timings is not None:
        timings["dense"] = t1 - t0
        timings["mvn"] = t2 - t1
    return n * math.log(2.0) + P.log_phi + lp, err


def loglik_batch(z, xy, thetas, tile: int = 128, tol: float = 1e-5, n_shifts: int = 10, n_points: int = 1000,
                 seed: int = 0, reorder: int = api.REORDER_BLOCK, timings=None):
    """log f(z; theta_k) for many parameter vectors, the MVN factors of all of them
    in one batched persistent launch (tlrmvn_prob_batch, float32 sweep; tiles of at
    most 128).  Returns (log f, err) arrays; problem k draws its lattice shifts from
    seed + k."""
    torch = _torch()
    n = len(z)
    t0 = time.perf_counter()
    D = distances(xy)
    logphi, Ss, bs = [], [], []
    for th in thetas:
        xi, s1, b1, s2, b2 = th
        A, B = model_matrices(D, s1, b1, s2, b2)
        P = parts(z, xi, A, B)
        logphi.append(P.log_phi)
        Ss.append(P.S.cpu().numpy())
        bs.append(P.bstar.cpu().numpy())
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    a = np.full(n, -np.inf)
    factors = [api.tlrmvn_factor_dense(S, a, b, tile, tol, 0, reorder) for S, b in zip(Ss, bs)]
    lp, err = api.tlrmvn_prob_batch(factors, [a] * len(factors), bs, math.inf, n_shifts, n_points, seed=seed)
    for F in factors:
        F.close()
    t2 = time.perf_counter()
    if timings is not None:
        timings["dense"] = t1 - t0
        timings["mvn"] = t2 - t1
    return n * math.log(2.0) + np.asarray(logphi) + lp, err


def simulate(xy, theta, seed: int) -> np.ndarray:
    """One draw of Z* = xi 1 + A X + B |Y| (eq. 5) at the locations (host float64)."""
    torch = _torch()
    xi, s1, b1, s2, b2 = theta
    A, B = model_matrices(distances(xy), s1, b1, s2, b2)
    rng = np.random.default_rng(seed)
    n = A.shape[0]
    X = torch.as_tensor(rng.standard_normal(n), device=A.device)
    Y = torch.as_tensor(np.abs(rng.standard_normal(n)), device=A.device)
    return (xi + A @ X + B @ Y).cpu().numpy()
