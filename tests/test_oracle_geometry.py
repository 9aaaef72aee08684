"""Pins for oracle.geometry: k-d indexing and covariance kernels."""
import math
import os
import numpy as np

from oracle import geometry
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_kd_order_quadrants_on_regular_grid():
    # 4x4 regular grid, m = 4: the leaves are the four 2x2 quadrants
    g = 4
    xy = np.array([[(i + 0.5) / g, (j + 0.5) / g] for i in range(g) for j in range(g)])
    perm, sizes = geometry.kd_order(xy, 4)
    assert list(sizes) == [4, 4, 4, 4]
    assert sorted(perm.tolist()) == list(range(16))
    quads = set()
    for t in range(4):
        pts = xy[perm[4 * t:4 * t + 4]]
        qx = set((pts[:, 0] > 0.5).tolist())
        qy = set((pts[:, 1] > 0.5).tolist())
        assert len(qx) == 1 and len(qy) == 1
        quads.add((qx.pop(), qy.pop()))
    assert len(quads) == 4
    # first split along x (equal extents -> x): first two leaves have x < 0.5
    assert np.all(xy[perm[:8], 0] < 0.5)


def test_kd_order_ragged_and_balanced():
    xy = synth.random_points(100, 3)
    perm, sizes = geometry.kd_order(xy, 16)
    assert list(sizes) == [16] * 6 + [4]
    assert sorted(perm.tolist()) == list(range(100))


def test_kd_leaves_are_spatially_separated():
    xy = synth.jittered_grid(16, 11)
    perm, sizes = geometry.kd_order(xy, 32)
    # every leaf's bounding box has area close to 32/256 of the square
    for t in range(len(sizes)):
        pts = xy[perm[32 * t:32 * (t + 1)]]
        ext = pts.max(0) - pts.min(0)
        assert ext[0] * ext[1] < 0.25


def test_exponential_effective_range_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "effective_range.txt")) if l.strip() and not l.startswith("#")]
    for beta, er in rows:
        c = geometry.kernel_value(float(er), geometry.KERNEL_EXP, (float(beta),))
        assert abs(c - math.exp(-3.0)) < 1e-12 and abs(c - 0.05) < 0.001


def test_kernels_closed_forms_and_spd():
    d = np.array([0.0, 0.1, 0.5])
    assert np.allclose(geometry.kernel_value(d, geometry.KERNEL_EXP, (0.1,)), np.exp(-d / 0.1))
    t = math.sqrt(3) * d / 0.2
    assert np.allclose(geometry.kernel_value(d, geometry.KERNEL_MATERN15, (0.2,)), (1 + t) * np.exp(-t))
    assert np.allclose(geometry.kernel_value(d, geometry.KERNEL_EXP_MATERN15, (0.3, 0.2)),
                       np.exp(-d / 0.3) + (1 + t) * np.exp(-t))
    xy = synth.jittered_grid(8, 2)
    for k, p in ((0, (0.1,)), (1, (0.1,)), (2, (0.3, 0.1))):
        S = geometry.covariance(xy, k, p, 1e-8)
        assert np.allclose(S, S.T)
        assert np.linalg.eigvalsh(S).min() > 0
        assert np.allclose(np.diag(S), (2.0 if k == 2 else 1.0) + 1e-8)
