"""Geometric indexing and covariance kernels (oracle; test infrastructure only).

Section 3.2: the covariance comes from spatial locations and a kernel; the
locations are indexed by a cardinality-balanced geometric partition whose
leaves (clusters) have the tile size m and become the TLR tiles.  The paper
uses HLIBpro's clustering; this is the reading adopted here, a k-d bisection:

* a set that spans t = ceil(size/m) tiles is split into the first ceil(t/2)*m
  points and the rest, so every leaf but the last holds exactly m points;
* the split runs along the coordinate with the larger extent (x on a tie);
* points are ranked by (that coordinate, the other coordinate, original index);
* leaves are visited depth first, left before right.

Kernels (Section 3.2, Table 2 caption; Section 3.2 on the Matern family):
exponential exp(-d/beta); Matern smoothness 3/2, (1 + sqrt3 d/ell) exp(-sqrt3 d/ell);
and their sum, each with unit variance.  A nugget is added on the diagonal.
"""
from __future__ import annotations

import math
import numpy as np

KERNEL_EXP = 0
KERNEL_MATERN15 = 1
KERNEL_EXP_MATERN15 = 2


def kd_order(xy: np.ndarray, m: int):
    """Returns (perm, tile_sizes): perm[position] = original index; leaves of size m (last ragged)."""
    xy = np.asarray(xy, dtype=np.float64)
    n = xy.shape[0]
    leaves = []

    def split(idx: np.ndarray):
        t = -(-idx.size // m)
        if t <= 1:
            leaves.append(idx)
            return
        nl = (-(-t // 2)) * m
        pts = xy[idx]
        ext = pts.max(axis=0) - pts.min(axis=0)
        axis = 0 if ext[0] >= ext[1] else 1
        other = 1 - axis
        rank = np.lexsort((idx, pts[:, other], pts[:, axis]))
        srt = idx[rank]
        split(srt[:nl])
        split(srt[nl:])

    split(np.arange(n, dtype=np.int64))
    perm = np.concatenate(leaves) if leaves else np.zeros(0, dtype=np.int64)
    return perm, np.array([lf.size for lf in leaves], dtype=np.int64)


def kernel_value(d: np.ndarray, kernel: int, params) -> np.ndarray:
    """Covariance as a function of distance d."""
    d = np.asarray(d, dtype=np.float64)
    if kernel == KERNEL_EXP:
        (beta,) = params[:1]
        return np.exp(-d / beta)
    if kernel == KERNEL_MATERN15:
        (ell,) = params[:1]
        t = math.sqrt(3.0) * d / ell
        return (1.0 + t) * np.exp(-t)
    if kernel == KERNEL_EXP_MATERN15:
        beta, ell = params[:2]
        t = math.sqrt(3.0) * d / ell
        return np.exp(-d / beta) + (1.0 + t) * np.exp(-t)
    raise ValueError(f"unknown kernel {kernel}")


def covariance(xy: np.ndarray, kernel: int, params, nugget: float, rows=None, cols=None) -> np.ndarray:
    """Sigma[rows][:, cols] with Sigma_ij = k(|x_i - x_j|) + nugget * [i == j]."""
    xy = np.asarray(xy, dtype=np.float64)
    ri = np.arange(xy.shape[0]) if rows is None else np.asarray(rows)
    ci = np.arange(xy.shape[0]) if cols is None else np.asarray(cols)
    dx = xy[ri, 0][:, None] - xy[ci, 0][None, :]
    dy = xy[ri, 1][:, None] - xy[ci, 1][None, :]
    d = np.sqrt(dx * dx + dy * dy)
    out = kernel_value(d, kernel, params)
    out = out + nugget * (ri[:, None] == ci[None, :])
    return out
