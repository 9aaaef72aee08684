"""Seeded synthetic inputs for the TLR quasi-Monte Carlo workloads.

This module is the only code shared by the CPU oracle (``oracle/``) and the
GPU library's tests and benchmark.  It holds no arithmetic of the method
itself: it only draws locations, integration limits, random lattice shifts and
kernel parameters from fixed seeds, with the shapes and distributions of the
paper's spatial workloads (Section 4: locations on a perturbed grid in the
unit square; lower limits at minus infinity; iid upper limits).

Seeds: grid jitter 1000+c, limits 2000+c, lattice shifts 3000+c for workload
number c, so every run sees the same inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
import numpy as np

KERNEL_EXP = 0          # sigma^2 exp(-d/beta)
KERNEL_MATERN15 = 1     # sigma^2 (1 + sqrt3 d/ell) exp(-sqrt3 d/ell)
KERNEL_EXP_MATERN15 = 2  # sum of the two, each with unit variance


def jittered_grid(g: int, seed: int, jitter: float = 0.8) -> np.ndarray:
    """g*g locations in the unit square: ((i + jitter*U)/g, (j + jitter*U)/g).

    Mirrors the paper's perturbed grid (Section 5.1 perturbs a regular grid by
    U(0, 0.8 * spacing)), rescaled so that the grid spans the unit square.
    Row-major enumeration: point index = i*g + j.  Returns float64 (g*g, 2).
    """
    rng = np.random.default_rng(seed)
    ii, jj = np.meshgrid(np.arange(g, dtype=np.float64), np.arange(g, dtype=np.float64), indexing="ij")
    u = rng.random((g * g, 2))
    xy = np.empty((g * g, 2), dtype=np.float64)
    xy[:, 0] = (ii.reshape(-1) + jitter * u[:, 0]) / g
    xy[:, 1] = (jj.reshape(-1) + jitter * u[:, 1]) / g
    return xy


def expanding_grid(g: int, spacing: float, seed: int, jitter: float = 0.8) -> np.ndarray:
    """g*g locations on a grid of the given spacing perturbed by U(0, jitter * spacing)
    per axis (Section 5.1: spacing 1/15, so the domain grows with n).  Returns (g*g, 2)."""
    rng = np.random.default_rng(seed)
    ii, jj = np.meshgrid(np.arange(g, dtype=np.float64), np.arange(g, dtype=np.float64), indexing="ij")
    u = rng.random((g * g, 2))
    xy = np.empty((g * g, 2), dtype=np.float64)
    xy[:, 0] = (ii.reshape(-1) + jitter * u[:, 0]) * spacing
    xy[:, 1] = (jj.reshape(-1) + jitter * u[:, 1]) * spacing
    return xy


def random_points(n: int, seed: int) -> np.ndarray:
    """n iid uniform locations in the unit square (for ragged, non-square n)."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 2))


def limits_uniform(n: int, seed: int, lo: float = 0.0, hi: float = 1.0):
    """a = -inf, b_i ~ U(lo, hi) iid."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(lo, hi, size=n)
    a = np.full(n, -np.inf)
    return a, b


def limits_normal(n: int, seed: int, mean: float, sd: float):
    """a = -inf, b_i ~ N(mean, sd^2) iid (the paper's Table 3 / Fig. 3 style)."""
    rng = np.random.default_rng(seed)
    b = rng.normal(mean, sd, size=n)
    a = np.full(n, -np.inf)
    return a, b


def lattice_shifts(n_shifts: int, n_coords: int, seed: int) -> np.ndarray:
    """Random shifts of the Richtmyer lattice as uint64 fixed-point fractions.

    Shape (n_shifts, n_coords); entry (s, i) is the shift of coordinate i in
    batch s, i.e. the fraction shift/2^64.  The method draws these at random;
    they are passed to both implementations as inputs.
    """
    rng = np.random.default_rng(seed)
    return rng.integers(0, np.iinfo(np.uint64).max, size=(n_shifts, n_coords), dtype=np.uint64, endpoint=True)


@dataclass
class Workload:
    """One synthetic MVN/MVT problem: geometry, kernel, limits, tiling, QMC sizes."""
    name: str
    xy: np.ndarray
    kernel: int
    params: tuple          # (beta) | (ell) | (beta, ell)
    nugget: float
    a: np.ndarray
    b: np.ndarray
    m: int
    tol: float
    max_rank: int
    nu: float              # math.inf for MVN
    n_shifts: int
    n_points: int
    shifts: np.ndarray = field(repr=False)
    reorder: int = 2       # 0 none, 1 block reordering, 2 iterative block reordering

    @property
    def n(self) -> int:
        return self.xy.shape[0]


def workload(c: int, n_side: int | None = None) -> Workload:
    """The five workload shapes, numbered 1..5, at full size.

    1: MVN n=256, 16x16 grid, exp beta=0.1, nugget 1e-8, b~U(0,1), m=64, tol 1e-8, 20x500, FP64
    2: MVN n=16,384, 128x128 grid, exp beta=0.3 + Matern 1.5 ell=0.1, b~U(0,1), m=256, tol 1e-5, 20x5000
    3: MVT nu=7, n=65,536, 256x256 grid, exp beta=0.1, b~N(1,0.5^2), m=512, tol 1e-4, rank<=64, 20x5000
    n_side (workload 3 only): a smaller grid of the same family, for profiling captures.
    """
    if c == 1:
        xy = jittered_grid(16, 1000 + c)
        a, b = limits_uniform(256, 2000 + c)
        return Workload("mvn_n256_exp", xy, KERNEL_EXP, (0.1,), 1e-8, a, b, 64, 1e-8, 64,
                        math.inf, 20, 500, lattice_shifts(20, 257, 3000 + c), reorder=2)
    if c == 2:
        xy = jittered_grid(128, 1000 + c)
        a, b = limits_uniform(16384, 2000 + c)
        return Workload("mvn_n16384_expmatern", xy, KERNEL_EXP_MATERN15, (0.3, 0.1), 1e-8, a, b, 256, 1e-5, 256,
                        math.inf, 20, 5000, lattice_shifts(20, 16385, 3000 + c), reorder=2)
    if c == 3:
        g = 256 if n_side is None else n_side
        xy = jittered_grid(g, 1000 + c)
        a, b = limits_normal(g * g, 2000 + c, 1.0, 0.5)
        name = "mvt7_n65536_exp" if g == 256 else f"mvt7_n{g * g}_exp"
        return Workload(name, xy, KERNEL_EXP, (0.1,), 1e-8, a, b, 512, 1e-4, 64,
                        7.0, 20, 5000, lattice_shifts(20, g * g + 1, 3000 + c), reorder=1)
    raise ValueError(f"unknown workload {c}")


def small_workload(n_side: int, m: int, seed: int, kernel: int = KERNEL_EXP, params=(0.1,), nu: float = math.inf,
                   n_shifts: int = 4, n_points: int = 64, tol: float = 1e-8, max_rank: int = 0,
                   limits: str = "uniform", reorder: int = 2, ragged_n: int | None = None) -> Workload:
    """A scaled-down problem of the same family, for parity tests the oracle finishes in seconds.

    ragged_n: if given, use that many uniform random points instead of a square grid
    (so that n is not a multiple of the tile size).
    """
    if ragged_n is not None:
        xy = random_points(ragged_n, 1000 + seed)
    else:
        xy = jittered_grid(n_side, 1000 + seed)
    n = xy.shape[0]
    if limits == "uniform":
        a, b = limits_uniform(n, 2000 + seed)
    elif limits == "normal":
        a, b = limits_normal(n, 2000 + seed, 1.0, 0.5)
    elif limits == "twosided":
        rng = np.random.default_rng(2000 + seed)
        lo = rng.uniform(-2.0, 0.5, size=n)
        a, b = lo, lo + rng.uniform(0.5, 3.0, size=n)
    else:
        raise ValueError(limits)
    return Workload(f"small_{n}_{m}_{seed}", xy, kernel, tuple(params), 1e-8, a, b, m, tol,
                    max_rank if max_rank > 0 else m, nu, n_shifts, n_points,
                    lattice_shifts(n_shifts, n + 1, 3000 + seed), reorder=reorder)


def batched_problems(count: int = 256, seed: int = 4000, n_min: int = 256, n_max: int = 4096):
    """The batched workload: `count` MVN problems, n log-uniform in [n_min, n_max], each
    with its own jittered grid (the first n points of a ceil(sqrt n)^2 grid), exponential
    kernel with beta ~ U(0.05, 0.3), b_i ~ U(0, 1).  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=count)).astype(int)
    betas = rng.uniform(0.05, 0.3, size=count)
    out = []
    for p in range(count):
        n = int(ns[p])
        g = int(math.ceil(math.sqrt(n)))
        xy = jittered_grid(g, seed + 1 + p)[:n]
        a, b = limits_uniform(n, seed + 10_000 + p)
        out.append({"xy": xy, "beta": float(betas[p]), "a": a, "b": b})
    return out
