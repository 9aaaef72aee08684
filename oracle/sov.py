"""SOV integrands and the QMC estimator (oracle; test infrastructure only).

* ``mvn_dense``: the dense integrand of eq. (2), i.e. Algorithm 1 with its two
  typesetting slips read from eq. (2): the divisor is the diagonal entry l_ii
  of the Cholesky factor, and y_i = Phi^-1(d_i + w_i (e_i - d_i)) with
  d_i = Phi(a'), e_i = Phi(b').
* ``tlrmvn``: Algorithm 6, the TLR integrand: after tile i-1 the limits of
  every later tile j are shifted by U_{j,i-1}(V_{j,i-1}^T y_{i-1}), then the
  dense integrand runs on diagonal tile B_i.
* ``mvt`` variants: Algorithms 3 and 7, which scale both limits by
  chi_nu^-1(w0)/sqrt(nu) and call the normal integrand.
* ``estimate``: Section 2.1 / Section 4: the estimate is the mean over the
  random-shift batches of the per-batch QMC means; its error is the standard
  error of that mean.  Everything is kept in logs because the probabilities
  underflow in high dimension (Section 4: likelihoods below 1e-40).

All integrands work on many samples at once: arrays are (variables, samples)
and every sample follows exactly the paper's per-sample recursion.
Samples are shift-major: sample s * N + (k - 1) is point k of shift batch s.
Lattice coordinate t drives the variable at position t; a Student-t problem
takes w0 from coordinate n.
"""
from __future__ import annotations

import math
import numpy as np
from scipy.special import logsumexp

from . import special
from . import lattice
from .factor import TLRFactor


def mvn_dense(L: np.ndarray, A: np.ndarray, Bm: np.ndarray, W: np.ndarray):
    """Eq. (2) / Algorithm 1 over samples.

    L: (n, n) lower Cholesky factor.  A, Bm: limits, (n, S) (or broadcastable).
    W: (n, S) lattice values.  Returns (logP (S,), Y (n, S)).
    """
    n = L.shape[0]
    S = W.shape[1]
    A = np.broadcast_to(A, (n, S))
    Bm = np.broadcast_to(Bm, (n, S))
    Y = np.zeros((n, S))
    logP = np.zeros(S)
    for i in range(n):
        s = L[i, :i] @ Y[:i] if i > 0 else np.zeros(S)
        with np.errstate(invalid="ignore"):
            at = (A[i] - s) / L[i, i]
            bt = (Bm[i] - s) / L[i, i]
        ld, y = special.sov_step(at, bt, W[i])
        Y[i] = y
        logP += ld
    return logP, Y


def tlrmvn(F: TLRFactor, A: np.ndarray, Bm: np.ndarray, W: np.ndarray):
    """Algorithm 6 over samples.  A, Bm, W: (n, S) in factor (permuted) order."""
    n = F.n
    S = W.shape[1]
    A = np.array(np.broadcast_to(A, (n, S)), dtype=np.float64, copy=True)
    Bm = np.array(np.broadcast_to(Bm, (n, S)), dtype=np.float64, copy=True)
    o = F.tile_off
    logP = np.zeros(S)
    y_prev = None
    for i in range(F.r):
        if i > 0:
            for j in range(i, F.r):
                delta = F.U[(j, i - 1)] @ (F.V[(j, i - 1)].T @ y_prev)
                A[o[j]:o[j + 1]] -= delta
                Bm[o[j]:o[j + 1]] -= delta
        lp, y_prev = mvn_dense(F.B[i], A[o[i]:o[i + 1]], Bm[o[i]:o[i + 1]], W[o[i]:o[i + 1]])
        logP += lp
    return logP


def mvt_scale(nu: float, w0: np.ndarray) -> np.ndarray:
    """chi_nu^-1(w0) / sqrt(nu): the per-sample limit scale of Algorithms 3 and 7."""
    return special.chi_inv(nu, w0) / math.sqrt(nu)


def per_sample_logp(F: TLRFactor | None, L_dense: np.ndarray | None, perm: np.ndarray, a, b, nu: float,
                    Wall: np.ndarray) -> np.ndarray:
    """log of the integrand for each sample (Algorithm 6/7, or eq. (2)/Algorithm 3 when L_dense is given).

    a, b: limits in original order; perm: position -> original index.
    Wall: (S, n + 1) lattice values, coordinate n feeds w0 for Student-t.
    """
    n = len(perm)
    ap = np.asarray(a, dtype=np.float64)[perm][:, None]
    bp = np.asarray(b, dtype=np.float64)[perm][:, None]
    W = Wall[:, :n].T
    if math.isfinite(nu):
        r = mvt_scale(nu, Wall[:, n])[None, :]
        ap = ap * r
        bp = bp * r
    if L_dense is not None:
        return mvn_dense(L_dense, ap, bp, W)[0]
    return tlrmvn(F, ap, bp, W)


def estimate(logP: np.ndarray, n_shifts: int, n_points: int):
    """(log p_hat, err, per-shift log means) from per-sample log integrand values.

    ell_s = log((1/N) sum_k P_{s,k}); p_hat = (1/M) sum_s exp(ell_s);
    err = SD_s(exp(ell_s)) / (sqrt(M) p_hat), the relative standard error of
    p_hat, which is also the standard error of log p_hat to first order.
    """
    Lm = np.asarray(logP, dtype=np.float64).reshape(n_shifts, n_points)
    ell = logsumexp(Lm, axis=1) - math.log(n_points)
    logp = float(logsumexp(ell) - math.log(n_shifts))
    if n_shifts > 1 and np.isfinite(ell).any():
        e = np.exp(ell - ell.max())
        err = float(np.std(e, ddof=1) / math.sqrt(n_shifts) / e.mean())
    else:
        err = float("nan")
    return logp, err, ell


def solve(F: TLRFactor | None, a, b, nu: float, shifts: np.ndarray, n_points: int, periodize: bool = True,
          L_dense: np.ndarray | None = None, perm: np.ndarray | None = None, chunk: int = 4096,
          samples: np.ndarray | None = None):
    """Full QMC solve.  Returns dict(logp, err, per_shift, per_sample).

    samples: optional subset of sample indices (0 .. M*N-1) to evaluate alone;
    then only per_sample (for those indices) is returned.
    """
    perm = F.perm if perm is None else perm
    n = len(perm)
    M = shifts.shape[0]
    Q = lattice.richtmyer_generators(n + 1)
    if samples is not None:
        samples = np.asarray(samples, dtype=np.int64)
        out = np.empty(samples.size)
        for c0 in range(0, samples.size, chunk):
            sel = samples[c0:c0 + chunk]
            s_idx, k_idx = np.divmod(sel, n_points)
            k = (k_idx + 1).astype(np.uint64)[:, None]
            with np.errstate(over="ignore"):
                x = k * Q[None, :] + shifts[s_idx]
            Wall = lattice.to_unit(x, periodize)
            out[c0:c0 + chunk] = per_sample_logp(F, L_dense, perm, a, b, nu, Wall)
        return {"per_sample": out}
    per_sample = np.empty(M * n_points)
    for s in range(M):
        x = lattice.lattice_u64(Q, shifts[s], n_points)
        Wall_s = lattice.to_unit(x, periodize)
        for c0 in range(0, n_points, chunk):
            per_sample[s * n_points + c0: s * n_points + min(n_points, c0 + chunk)] = \
                per_sample_logp(F, L_dense, perm, a, b, nu, Wall_s[c0:c0 + chunk])
    logp, err, ell = estimate(per_sample, M, n_points)
    return {"logp": logp, "err": err, "per_shift": ell, "per_sample": per_sample}
