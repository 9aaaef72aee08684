"""Test utilities: convert factors between the library's export layout and the oracle."""
from __future__ import annotations

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
