"""Test utilities: convert factors between the library's export layout and the oracle."""
from __future__ import annotations

import math

import numpy as np

from oracle import factor as ofactor, geometry


def to_oracle_factor(ex) -> ofactor.TLRFactor:
    """An oracle TLRFactor holding exactly the arrays of an exported library factor."""
    sizes = np.diff(ex.tile_off)
    B = [ex.B[t, :sizes[t], :sizes[t]].copy() for t in range(ex.r)]
    U, V = {}, {}
    for i in range(ex.r):
        for j in range(i):
            if (i, j) in ex.U:
                U[(i, j)], V[(i, j)] = ex.U[(i, j)], ex.V[(i, j)]
            else:
                U[(i, j)], V[(i, j)] = np.zeros((sizes[i], 0)), np.zeros((sizes[j], 0))
    return ofactor.TLRFactor(ex.n, ex.m, ex.perm.copy(), ex.tile_off.copy(), B, U, V)


def oracle_factor(w, reorder=None):
    """The oracle's own factor of a synthetic workload (dense covariance; small n only)."""
    perm0, sizes = geometry.kd_order(w.xy, w.m)
    Sig = geometry.covariance(w.xy, w.kernel, w.params, w.nugget)
    F = ofactor.tlr_factor(Sig, perm0, sizes, w.a, w.b, w.tol, w.max_rank, w.reorder if reorder is None else reorder)
    return F, Sig


def export_bytes(F: ofactor.TLRFactor) -> bytes:
    from paper_2003_11183_gb300.api import build_export
    U = {k: v for k, v in F.U.items() if v.shape[1] > 0}
    V = {k: F.V[k] for k in U}
    return build_export(F.n, F.m, F.tile_off, F.perm, F.B, U, V)


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def factor_row(F: ofactor.TLRFactor, t: int) -> np.ndarray:
    """Row t (factor position) of the dense TLR factor L, without assembling L."""
    o = F.tile_off
    i = int(np.searchsorted(o, t, side="right") - 1)
    row = np.zeros(F.n)
    v = t - o[i]
    row[o[i]:o[i] + v + 1] = F.B[i][v, :v + 1]
    for j in range(i):
        U, V = F.U[(i, j)], F.V[(i, j)]
        if U.shape[1]:
            row[o[j]:o[j + 1]] = V @ U[v]
    return row


def sampled_reconstruction_error(F: ofactor.TLRFactor, xy, kernel, params, nugget, pairs) -> float:
    """max |(L L^T)[s, t] - Sigma[perm[s], perm[t]]| over the given position pairs."""
    rows = {}
    worst = 0.0
    for s, t in pairs:
        for q in (s, t):
            if q not in rows:
                rows[q] = factor_row(F, q)
        got = rows[s] @ rows[t]
        want = geometry.covariance(xy, kernel, params, nugget, rows=[F.perm[s]], cols=[F.perm[t]])[0, 0]
        worst = max(worst, abs(got - want))
    return worst


def sources_targets_factor(n: int, m: int, seed: int, max_rank: int = 3):
    """A TLR factor whose integrand has a closed form per sample, at any size.

    Tiles alternate: even tiles are sources (random dense lower-triangular B with
    positive diagonal; their limits will be infinite), odd tiles are targets
    (B = identity).  Every pair (later tile i, earlier tile j) has random low-rank
    factors U_ij, V_ij of rank 1..max_rank, except target-to-target pairs, which
    have rank 0.  With a = -inf everywhere, b = +inf on sources and finite b on
    targets, eq. 2 gives y = Phi^-1(w) on every source variable, a zero log term
    there, and on target variable v of tile i the term log Phi(b_v - s_v) with
    s = sum over sources j < i of U_ij V_ij^T Phi^-1(w_j) (see closed_form_logf).
    Returns (F, b) in factor order (perm = identity).
    """
    rng = np.random.default_rng(seed)
    r = n // m
    tile_off = np.arange(r + 1) * m
    B, U, V = [], {}, {}
    for t in range(r):
        if t % 2 == 0:
            Bt = np.tril(rng.normal(0.0, 0.3, (m, m)), -1)
            Bt[np.diag_indices(m)] = rng.uniform(0.5, 1.5, m)
        else:
            Bt = np.eye(m)
        B.append(Bt)
    n_src = (r + 1) // 2
    for i in range(r):
        for j in range(i):
            k = 0 if (i % 2 == 1 and j % 2 == 1) else int(rng.integers(1, max_rank + 1))
            U[(i, j)] = rng.normal(0.0, 1.0 / math.sqrt(max(1, k * n_src)), (m, k))
            V[(i, j)] = rng.normal(0.0, 1.0 / math.sqrt(m), (m, k))
    F = ofactor.TLRFactor(n, m, np.arange(n), tile_off, B, U, V)
    b = np.full(n, np.inf)
    for t in range(1, r, 2):
        b[t * m:(t + 1) * m] = rng.normal(1.0, 0.5, m)
    return F, b


def closed_form_logf(F: ofactor.TLRFactor, b: np.ndarray, W: np.ndarray, rs: np.ndarray | None = None) -> np.ndarray:
    """Per-sample log integrand of a sources_targets_factor problem, computed directly:
    sum over target variables of log Phi(r b_v - s_v), s as described there and r the
    sample's Student-t scale (rs, one per sample; 1 for a normal problem).  W: (n, S)."""
    from scipy.special import log_ndtr, ndtri
    o = F.tile_off
    r = np.ones(W.shape[1]) if rs is None else np.asarray(rs, dtype=np.float64)
    out = np.zeros(W.shape[1])
    Y = {j: ndtri(W[o[j]:o[j + 1]]) for j in range(0, F.r, 2)}
    for i in range(1, F.r, 2):
        s = np.zeros((o[i + 1] - o[i], W.shape[1]))
        for j in range(0, i, 2):
            s += F.U[(i, j)] @ (F.V[(i, j)].T @ Y[j])
        out += log_ndtr(b[o[i]:o[i + 1], None] * r[None, :] - s).sum(axis=0)
    return out
