"""Randomly shifted Richtmyer lattice (oracle; test infrastructure only).

Section 2.1: the integrand is averaged over a Richtmyer quasi-Monte Carlo rule,
with few random-shift batches of many points each; Section 3.4 repeats the
choice for the TLR integrand.  The Richtmyer rule takes the fractional parts of
k * sqrt(p_i) for the i-th prime p_i.  Here every fraction is an exact uint64
fixed-point number (fraction = x / 2^64), so that

    x_{s,k,i} = (k * Q_i + D_{s,i}) mod 2^64,   Q_i = floor(frac(sqrt(p_i)) * 2^64),

with k = 1..N the point index, s the shift batch and D the random shift.
Periodisation (the paper does not say; the baker's / tent transform of Genz &
Bretz, 2009) maps the point to w = |2x - 1|; all arithmetic stays exact by
working on the top 53 bits h = x >> 11 and the midpoint (h + 1/2) / 2^53.
"""
from __future__ import annotations

import math
import numpy as np

TWO53 = 1 << 53


def primes(count: int) -> np.ndarray:
    """The first ``count`` primes (2, 3, 5, ...) by the sieve of Eratosthenes."""
    if count <= 0:
        return np.zeros(0, dtype=np.int64)
    bound = 16
    while True:
        sieve = np.ones(bound + 1, dtype=bool)
        sieve[:2] = False
        for p in range(2, int(math.isqrt(bound)) + 1):
            if sieve[p]:
                sieve[p * p::p] = False
        ps = np.flatnonzero(sieve)
        if ps.size >= count:
            return ps[:count].astype(np.int64)
        bound *= 2


def richtmyer_generators(d: int) -> np.ndarray:
    """Q_i = floor(frac(sqrt(p_i)) * 2^64) for the first d primes, exactly (integer square root)."""
    out = np.empty(d, dtype=np.uint64)
    for i, p in enumerate(primes(d)):
        out[i] = math.isqrt(int(p) << 128) & ((1 << 64) - 1)
    return out


def lattice_u64(Q: np.ndarray, shift: np.ndarray, n_points: int) -> np.ndarray:
    """(n_points, d) uint64 fractions (k Q_i + D_i) mod 2^64 for k = 1..n_points."""
    k = np.arange(1, n_points + 1, dtype=np.uint64)[:, None]
    with np.errstate(over="ignore"):
        return k * Q[None, :] + shift[None, :]


def to_unit(x: np.ndarray, periodize: bool = True) -> np.ndarray:
    """Map uint64 fractions to w in (0, 1), exactly representable in float64.

    With the tent transform: h = x >> 11 (53 bits) and
    w = |2(h + 1/2)/2^53 - 1| = |2h + 1 - 2^53| / 2^53, an odd integer over 2^53.
    Without it: h = x >> 12 (52 bits) and w = (2h + 1) / 2^53, the midpoint of the
    h-th cell.  Either way the numerator is an odd integer below 2^53, so w is
    exact in float64 and never 0 or 1.
    """
    if periodize:
        h = (x >> np.uint64(11)).astype(np.int64)
        num = np.abs(2 * h + 1 - TWO53)
        return num.astype(np.float64) * (2.0 ** -53)
    h = (x >> np.uint64(12)).astype(np.int64)
    return (2 * h + 1).astype(np.float64) * (2.0 ** -53)


def qmc_points(Q: np.ndarray, shifts: np.ndarray, n_points: int, periodize: bool = True) -> np.ndarray:
    """All samples, shift-major: row s * n_points + (k - 1) holds point k of shift batch s."""
    blocks = [to_unit(lattice_u64(Q, shifts[s], n_points), periodize) for s in range(shifts.shape[0])]
    return np.concatenate(blocks, axis=0)
