"""Pins for oracle.lattice: primes, Richtmyer generators, fixed-point points, periodisation."""
from decimal import Decimal, getcontext
import numpy as np

from oracle import lattice


def test_primes():
    assert list(lattice.primes(10)) == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29]
    p = lattice.primes(70000)
    sympy = __import__("pytest").importorskip("sympy")
    assert p[-1] == sympy.prime(70000)
    assert p[65536] == sympy.prime(65537)  # the coordinate w0 of an n = 65,536 Student-t problem
    assert np.all(np.diff(p) > 0)


def test_generators_against_decimal_sqrt():
    # floor(frac(sqrt(p)) * 2^64) recomputed with 60-digit decimal arithmetic
    getcontext().prec = 60
    Q = lattice.richtmyer_generators(60)
    for i, p in enumerate(lattice.primes(60)):
        s = Decimal(int(p)).sqrt()
        frac = s - int(s)
        want = int(frac * (Decimal(2) ** 64))
        assert int(Q[i]) == want


def test_points_are_fixed_point_fractions():
    Q = lattice.richtmyer_generators(3)
    D = np.array([0, 5, 2**63], dtype=np.uint64)
    x = lattice.lattice_u64(Q, D, 4)
    for k in range(1, 5):
        for i in range(3):
            assert int(x[k - 1, i]) == (k * int(Q[i]) + int(D[i])) % 2**64


def test_unit_mapping_exact_and_open():
    x = np.array([0, 1, 2**11 - 1, 2**11, 2**63 - 1, 2**63, 2**64 - 1], dtype=np.uint64)
    w = lattice.to_unit(x, True)
    assert np.all((w > 0) & (w < 1))
    # tent transform of the cell midpoint, exactly
    for xi, wi in zip(x.tolist(), w.tolist()):
        h = xi >> 11
        assert wi == abs(2 * h + 1 - 2**53) / 2**53
    # tent symmetry: x and its complement 2^64 - 1 - x give the same w
    assert np.array_equal(lattice.to_unit(~x, True), w)
    w0 = lattice.to_unit(x, False)
    assert np.all((w0 > 0) & (w0 < 1))
    assert w0[0] == 2.0**-53 and w0[-1] == 1 - 2.0**-53


def test_qmc_rule_integrates_smooth_function():
    # mean of prod_i (1 + (w_i - 1/2)) over the shifted lattice ~ 1 (exact integral)
    Q = lattice.richtmyer_generators(8)
    rng = np.random.default_rng(5)
    D = rng.integers(0, 2**64 - 1, size=(4, 8), dtype=np.uint64, endpoint=True)
    W = lattice.qmc_points(Q, D, 4096)
    f = np.prod(1 + (W - 0.5), axis=1)
    assert abs(f.mean() - 1.0) < 2e-3
