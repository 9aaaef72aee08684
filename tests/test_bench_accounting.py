"""The algorithmic work the bench line's roofline divides by (bench.sweep_work), against its
closed forms: eq. 2 costs (mt - 1) flops per variable of a tile of mt variables (one FMA for each
earlier variable of the tile, averaged over the tile); the low-rank shifts and projections cost
2 m K_total flops each per sample; the split coupling between 64-variable sub-tiles issues three
products of 2 * 64 * q0 flops before sub-tile q0 / 64."""
import math

import bench


def test_sweep_work_bench_workload():
    n, m, ktot = 65_536, 512, 28_397
    w = bench.sweep_work(None, [m] * (n // m), m, ktot, n)
    assert w["sweep"] == m - 1
    assert math.isclose(w["shift_proj"], 4 * m * ktot / n)
    # per tile: 3 * 2 * 64 * (64 + 128 + ... + 448) = 6 * 64 * 64 * 28
    couple = (n // m) * 6 * 64 * 64 * 28 / n
    assert math.isclose(w["tensor"], 4 * m * ktot / n + couple)
    assert math.isclose(w["tensor"], 2231.40625)


def test_sweep_work_ragged_tiles():
    n, m = 1_000, 512
    sizes = [512, 488]
    w = bench.sweep_work(None, sizes, m, 0, n)
    assert math.isclose(w["sweep"], (512 * 511 + 488 * 487) / n)
    # sub-tiles of the 488-variable tile: q0 = 64 ... 448, the last one 40 variables
    couple = sum(6 * 64 * q0 for q0 in range(64, 512, 64)) + sum(6 * min(64, 488 - q0) * q0 for q0 in range(64, 488, 64))
    assert math.isclose(w["tensor"], couple / n)
    assert w["shift_proj"] == 0.0


def test_small_tiles_have_no_coupling_products():
    w = bench.sweep_work(None, [64] * 16, 64, 100, 1024)
    assert w["sweep"] == 63
    assert math.isclose(w["tensor"], 4 * 64 * 100 / 1024)
