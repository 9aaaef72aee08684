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


def _matern_bessel(d, nu, ell):
    """The general Matern covariance, 2^(1-nu)/Gamma(nu) x^nu K_nu(x) with x = sqrt(2 nu) d / ell
    (unit variance; the limit 1 at d = 0), from the modified Bessel function of the second kind."""
    from scipy.special import gamma, kv
    d = np.asarray(d, dtype=np.float64)
    x = math.sqrt(2.0 * nu) * d / ell
    with np.errstate(invalid="ignore"):
        out = 2.0 ** (1.0 - nu) / gamma(nu) * x ** nu * kv(nu, x)
    return np.where(d == 0.0, 1.0, out)


def test_kernels_equal_the_bessel_matern_family():
    # Section 3.2's kernels are members of the Matern family: the exponential kernel is
    # smoothness 1/2 with range beta, the "Matern 1.5" kernel smoothness 3/2 with range
    # ell in the sqrt(2 nu) d / ell convention; both pinned to the Bessel-K form, which
    # fixes the length-scale convention and every term of the closed forms
    d = np.concatenate([[0.0, 1e-9], np.geomspace(1e-4, 2.0, 41)])
    for ell in (0.05, 0.1, 0.2):
        got = geometry.kernel_value(d, geometry.KERNEL_MATERN15, (ell,))
        assert np.max(np.abs(got - _matern_bessel(d, 1.5, ell))) < 1e-13
        got = geometry.kernel_value(d, geometry.KERNEL_EXP, (ell,))
        assert np.max(np.abs(got - _matern_bessel(d, 0.5, ell))) < 1e-13
    got = geometry.kernel_value(d, geometry.KERNEL_EXP_MATERN15, (0.3, 0.1))
    want = _matern_bessel(d, 0.5, 0.3) + _matern_bessel(d, 1.5, 0.1)
    assert np.max(np.abs(got - want)) < 1e-13
    # a plausible slip is caught: the d / ell convention (without sqrt 3) differs by far more
    t = d / 0.1
    assert np.max(np.abs((1 + t) * np.exp(-t) - _matern_bessel(d, 1.5, 0.1))) > 1e-2


def test_kernels_spd():
    xy = synth.jittered_grid(8, 2)
    for k, p in ((0, (0.1,)), (1, (0.1,)), (2, (0.3, 0.1))):
        S = geometry.covariance(xy, k, p, 1e-8)
        assert np.allclose(S, S.T)
        assert np.linalg.eigvalsh(S).min() > 0
        assert np.allclose(np.diag(S), (2.0 if k == 2 else 1.0) + 1e-8)
