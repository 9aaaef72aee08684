"""Pins for oracle.sov: the dense and TLR integrands, Student-t scaling and the estimator.

Closed forms: n = 1; independent variables; bivariate and trivariate orthants
(normal and, by elliptical symmetry, Student-t); the univariate t CDF; infinite
limits; block-diagonal covariance; scale invariance.  Library routines: scipy's
multivariate normal CDF, adaptive quadrature.  Brute force: plain Monte Carlo.
"""
import math
import numpy as np
import pytest
from scipy import stats, integrate

from oracle import sov, factor, geometry, lattice, special
import synth


def _shifts(M, d, seed):
    return synth.lattice_shifts(M, d + 1, seed)


def _solve_dense(Sig, a, b, nu=math.inf, M=8, N=2000, seed=1, periodize=True):
    L = np.linalg.cholesky(Sig)
    n = Sig.shape[0]
    return sov.solve(None, a, b, nu, _shifts(M, n, seed), N, periodize, L_dense=L, perm=np.arange(n))


def test_n1_is_exact_for_every_sample():
    for a, b in [(-np.inf, 0.7), (-0.4, 1.1), (2.5, np.inf), (3.0, 6.0)]:
        res = _solve_dense(np.array([[2.25]]), np.array([a]), np.array([b]), M=2, N=50)
        want = math.log(stats.norm.cdf(b / 1.5) - stats.norm.cdf(a / 1.5))
        assert np.allclose(res["per_sample"], want, rtol=1e-13, atol=1e-14)
        assert abs(res["logp"] - want) < 1e-12


def test_independent_variables_exact_product():
    rng = np.random.default_rng(2)
    n = 20
    sd = rng.uniform(0.5, 2, n)
    a = np.where(rng.random(n) < 0.5, -np.inf, rng.uniform(-2, 0, n))
    b = rng.uniform(0.1, 2, n)
    want = np.sum(np.log(stats.norm.cdf(b / sd) - stats.norm.cdf(a / sd)))
    res = _solve_dense(np.diag(sd**2), a, b, M=3, N=40)
    assert np.allclose(res["per_sample"], want, rtol=1e-12)
    # TLR path on the same problem (tiles of 6, ranks 0)
    F = factor.tlr_factor(np.diag(sd**2), np.arange(n), [6, 6, 6, 2], a, b, 1e-10, 6, 2)
    res2 = sov.solve(F, a, b, math.inf, _shifts(3, n, 4), 40)
    assert np.allclose(res2["per_sample"], want, rtol=1e-12)


@pytest.mark.parametrize("nu", [math.inf, 3.0, 7.0])
def test_bivariate_orthant(nu):
    for rho in (-0.7, 0.3, 0.9):
        Sig = np.array([[1.0, rho], [rho, 1.0]])
        z = np.zeros(2)
        res = _solve_dense(Sig, np.full(2, -np.inf), z, nu=nu, M=10, N=4000)
        want = 0.25 + math.asin(rho) / (2 * math.pi)
        p = math.exp(res["logp"])
        assert abs(p - want) <= 4 * res["err"] * p + 1e-6, (rho, nu, p, want)


@pytest.mark.parametrize("nu", [math.inf, 5.0])
def test_trivariate_orthant(nu):
    R = np.array([[1.0, 0.5, 0.3], [0.5, 1.0, -0.2], [0.3, -0.2, 1.0]])
    res = _solve_dense(R, np.full(3, -np.inf), np.zeros(3), nu=nu, M=10, N=4000)
    want = 0.125 + (math.asin(0.5) + math.asin(0.3) + math.asin(-0.2)) / (4 * math.pi)
    p = math.exp(res["logp"])
    assert abs(p - want) <= 4 * res["err"] * p + 1e-6


def test_student_t_univariate_cdf():
    for nu in (3.0, 7.0):
        for a, b in [(-np.inf, 0.8), (-1.0, 2.0), (1.5, np.inf)]:
            res = _solve_dense(np.array([[4.0]]), np.array([a]), np.array([b]), nu=nu, M=10, N=4000)
            want = stats.t.cdf(b / 2, nu) - stats.t.cdf(a / 2, nu)
            p = math.exp(res["logp"])
            assert abs(p - want) <= 4 * res["err"] * p + 1e-9, (nu, a, b, p, want)


def test_infinite_limits_give_zero_log():
    xy = synth.jittered_grid(4, 1)
    Sig = geometry.covariance(xy, 0, (0.2,), 1e-8)
    res = _solve_dense(Sig, np.full(16, -np.inf), np.full(16, np.inf), M=2, N=20)
    assert np.all(res["per_sample"] == 0.0)


def test_block_diagonal_factorises_per_sample():
    # two independent blocks: each sample's log integrand is the sum of the two
    # block integrands fed with the same lattice coordinates
    rng = np.random.default_rng(3)
    A1 = rng.normal(size=(5, 5)); S1 = A1 @ A1.T + 5 * np.eye(5)
    A2 = rng.normal(size=(4, 4)); S2 = A2 @ A2.T + 4 * np.eye(4)
    Sig = np.zeros((9, 9)); Sig[:5, :5] = S1; Sig[5:, 5:] = S2
    a = np.full(9, -np.inf); b = rng.uniform(0, 3, 9)
    Q = lattice.richtmyer_generators(10)
    W = lattice.qmc_points(Q, _shifts(3, 9, 7), 64).T
    full, _ = sov.mvn_dense(np.linalg.cholesky(Sig), a[:, None], b[:, None], W[:9])
    p1, _ = sov.mvn_dense(np.linalg.cholesky(S1), a[:5, None], b[:5, None], W[:5])
    p2, _ = sov.mvn_dense(np.linalg.cholesky(S2), a[5:, None], b[5:, None], W[5:9])
    assert np.allclose(full, p1 + p2, rtol=1e-12)
    # and the TLR factor of it has zero-rank off-diagonal tiles
    F = factor.tlr_factor(Sig, np.arange(9), [5, 4], a, b, 1e-12, 5, 0)
    assert F.rank(1, 0) == 0


def test_scale_invariance_per_sample():
    xy = synth.jittered_grid(5, 6)
    Sig = geometry.covariance(xy, 0, (0.3,), 1e-8)
    a, b = synth.limits_uniform(25, 8)
    dsc = np.linspace(0.5, 3.0, 25)
    r1 = _solve_dense(Sig, a, b, M=2, N=50)
    r2 = _solve_dense(Sig * np.outer(dsc, dsc), a * dsc, b * dsc, M=2, N=50)
    assert np.allclose(r1["per_sample"], r2["per_sample"], rtol=1e-10)


def test_against_scipy_mvn_cdf_and_plain_monte_carlo():
    rng = np.random.default_rng(4)
    n = 6
    xy = rng.random((n, 2))
    Sig = geometry.covariance(xy, 0, (0.5,), 1e-8)
    b = rng.uniform(0.0, 1.5, n)
    a = np.full(n, -np.inf)
    res = _solve_dense(Sig, a, b, M=10, N=5000)
    p = math.exp(res["logp"])
    ref = stats.multivariate_normal(mean=np.zeros(n), cov=Sig).cdf(b)
    assert abs(p - ref) <= 4 * res["err"] * p + 1e-4
    X = rng.multivariate_normal(np.zeros(n), Sig, size=2_000_000)
    hit = np.all(X <= b, axis=1)
    pm, sm = hit.mean(), hit.std() / math.sqrt(hit.size)
    assert abs(p - pm) <= 4 * math.hypot(sm, res["err"] * p)


def test_bivariate_rectangle_against_quadrature():
    rho = 0.6
    Sig = np.array([[1.0, rho], [rho, 1.0]])
    a = np.array([-0.5, -1.0]); b = np.array([1.2, 0.4])
    s = math.sqrt(1 - rho**2)
    f = lambda x: stats.norm.pdf(x) * (stats.norm.cdf((b[1] - rho * x) / s) - stats.norm.cdf((a[1] - rho * x) / s))
    want, _ = integrate.quad(f, a[0], b[0], epsabs=1e-13, epsrel=1e-13)
    res = _solve_dense(Sig, a, b, M=10, N=4000)
    p = math.exp(res["logp"])
    assert abs(p - want) <= 4 * res["err"] * p + 1e-8
    assert res["err"] < 1e-3


def _tlr_case(seed, reorder=2, tol=1e-8, ragged=None, nu=math.inf, m=32, n_side=16):
    w = synth.small_workload(n_side, m, seed, tol=tol, ragged_n=ragged, nu=nu, n_shifts=3, n_points=64)
    perm0, sizes = geometry.kd_order(w.xy, w.m)
    Sig = geometry.covariance(w.xy, w.kernel, w.params, w.nugget)
    F = factor.tlr_factor(Sig, perm0, sizes, w.a, w.b, w.tol, w.max_rank, reorder)
    return w, Sig, F


@pytest.mark.parametrize("nu", [math.inf, 7.0])
@pytest.mark.parametrize("ragged", [None, 200])
def test_tlr_recursion_equals_dense_recursion_on_same_factor(nu, ragged):
    # Algorithm 6 on (B, U, V) and eq. (2) on the assembled dense factor are the same sums
    w, Sig, F = _tlr_case(21, ragged=ragged, nu=nu)
    r1 = sov.solve(F, w.a, w.b, nu, w.shifts, w.n_points)
    r2 = sov.solve(None, w.a, w.b, nu, w.shifts, w.n_points, L_dense=F.dense(), perm=F.perm)
    assert np.allclose(r1["per_sample"], r2["per_sample"], rtol=1e-11, atol=1e-11)


def test_tlr_at_tight_tolerance_matches_exact_cholesky():
    w, Sig, F = _tlr_case(22, tol=1e-8)
    P = F.perm
    Ld = np.linalg.cholesky(Sig[np.ix_(P, P)])
    r1 = sov.solve(F, w.a, w.b, math.inf, w.shifts, w.n_points)
    r2 = sov.solve(None, w.a, w.b, math.inf, w.shifts, w.n_points, L_dense=Ld, perm=P)
    assert np.abs(r1["per_sample"] - r2["per_sample"]).max() < 1e-5
    assert abs(r1["logp"] - r2["logp"]) < 1e-6


def test_tlr_1024_tol_1e8_close_to_dense():
    w, Sig, F = _tlr_case(23, tol=1e-8, m=128, n_side=32)
    P = F.perm
    Ld = np.linalg.cholesky(Sig[np.ix_(P, P)])
    sel = np.arange(0, w.n_shifts * w.n_points, 7)
    r1 = sov.solve(F, w.a, w.b, math.inf, w.shifts, w.n_points, samples=sel)
    r2 = sov.solve(None, w.a, w.b, math.inf, w.shifts, w.n_points, L_dense=Ld, perm=P, samples=sel)
    assert np.abs(r1["per_sample"] - r2["per_sample"]).max() < 1e-5


def test_reordering_leaves_the_estimate_unchanged():
    w, Sig, F0 = _tlr_case(24, reorder=0, m=16, n_side=8)
    _, _, F2 = _tlr_case(24, reorder=2, m=16, n_side=8)
    D = synth.lattice_shifts(10, w.n + 1, 99)
    r0 = sov.solve(F0, w.a, w.b, math.inf, D, 1000)
    r2 = sov.solve(F2, w.a, w.b, math.inf, D, 1000)
    assert abs(r0["logp"] - r2["logp"]) <= 3 * math.hypot(r0["err"], r2["err"])


def test_estimator_closed_forms():
    lp = np.full(12, -3.5)
    logp, err, ell = sov.estimate(lp, 3, 4)
    assert abs(logp + 3.5) < 1e-14 and err == 0.0
    # two shifts with per-shift means 1/4 and 3/4 (in probability): p_hat = 1/2,
    # SD = sqrt(1/8), err = SD/(sqrt(2) p_hat) = 1/2
    lp = np.log(np.array([0.25, 0.25, 0.5, 1.0]))
    logp, err, ell = sov.estimate(lp, 2, 2)
    assert abs(logp - math.log(0.5)) < 1e-14
    assert abs(err - 0.5) < 1e-14
