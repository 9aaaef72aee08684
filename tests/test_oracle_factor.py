"""Pins for oracle.factor: univariate conditioning, ACA, block reorderings, TLR Cholesky."""
import math
import numpy as np
import pytest
from scipy import stats

from oracle import factor, geometry, special
import synth


def test_uc_one_variable():
    for a, b in [(-np.inf, 0.3), (-1.0, 0.5), (2.0, np.inf)]:
        r = factor.univariate_conditioning(np.array([[4.0]]), np.array([a]), np.array([b]))
        want = math.log(stats.norm.cdf(b / 2) - stats.norm.cdf(a / 2))
        assert abs(r.log_p - want) < 1e-13
        assert abs(r.y[0] - stats.truncnorm.mean(a / 2, b / 2)) < 1e-10
        assert r.L[0, 0] == 2.0


def test_uc_diagonal_is_exact_and_sorted():
    rng = np.random.default_rng(0)
    sd = rng.uniform(0.5, 2.0, 12)
    b = rng.uniform(-1, 2, 12)
    a = np.full(12, -np.inf)
    r = factor.univariate_conditioning(np.diag(sd**2), a, b)
    q = stats.norm.logcdf(b / sd)
    assert np.array_equal(r.order, np.argsort(q, kind="stable"))
    assert abs(r.log_p - q.sum()) < 1e-12
    assert np.allclose(np.diag(r.L), sd[r.order])


def test_uc_bivariate_by_hand():
    S = np.array([[1.0, 0.6], [0.6, 2.0]])
    a = np.array([-np.inf, -np.inf])
    b = np.array([1.5, 0.2])
    r = factor.univariate_conditioning(S, a, b)
    # Phi(1.5) > Phi(0.2/sqrt2): variable 1 first
    assert list(r.order) == [1, 0]
    l11 = math.sqrt(2.0)
    y1 = stats.truncnorm.mean(-np.inf, 0.2 / l11)
    l21 = 0.6 / l11
    l22 = math.sqrt(1.0 - l21**2)
    want = stats.norm.logcdf(0.2 / l11) + stats.norm.logcdf((1.5 - l21 * y1) / l22)
    assert abs(r.log_p - want) < 1e-12
    assert np.allclose(r.L, [[l11, 0], [l21, l22]])


def test_uc_factor_reproduces_permuted_covariance():
    xy = synth.jittered_grid(6, 4)
    S = geometry.covariance(xy, 0, (0.2,), 1e-8)
    a, b = synth.limits_uniform(36, 9)
    r = factor.univariate_conditioning(S, a, b)
    assert np.allclose(r.L @ r.L.T, S[np.ix_(r.order, r.order)], atol=1e-12)
    assert sorted(r.order) == list(range(36))


def test_aca_exact_low_rank_and_tolerance():
    rng = np.random.default_rng(1)
    A = rng.normal(size=(40, 3)) @ rng.normal(size=(3, 30))
    U, V, capped = factor.aca(A, 1e-10, 40)
    assert U.shape[1] == 3 and not capped
    assert np.abs(A - U @ V.T).max() < 1e-10
    # tolerance bound on a decaying kernel block
    xy = synth.jittered_grid(8, 1)
    B = geometry.covariance(xy, 0, (0.3,), 0.0, rows=np.arange(32), cols=np.arange(32, 64))
    for tol in (1e-2, 1e-4, 1e-8):
        U, V, capped = factor.aca(B, tol, 64)
        assert np.abs(B - U @ V.T).max() <= tol
    # zero block -> rank 0; cap flag
    U, V, capped = factor.aca(np.zeros((5, 4)), 1e-8, 3)
    assert U.shape == (5, 0) and V.shape == (4, 0) and not capped
    U, V, capped = factor.aca(rng.normal(size=(6, 6)), 1e-12, 2)
    assert U.shape[1] == 2 and capped
    # balanced terms
    U, V, _ = factor.aca(A, 1e-10, 40)
    assert np.allclose(np.linalg.norm(U, axis=0), np.linalg.norm(V, axis=0))


def _factor(n_side, m, seed, reorder, tol=1e-8, ragged=None, kernel=0, params=(0.1,)):
    w = synth.small_workload(n_side, m, seed, kernel=kernel, params=params, ragged_n=ragged, tol=tol)
    perm0, sizes = geometry.kd_order(w.xy, w.m)
    Sig = geometry.covariance(w.xy, w.kernel, w.params, w.nugget)
    F = factor.tlr_factor(Sig, perm0, sizes, w.a, w.b, w.tol, w.max_rank, reorder)
    return w, Sig, F


@pytest.mark.parametrize("reorder", [0, 1, 2])
@pytest.mark.parametrize("ragged", [None, 200])
def test_tlr_factor_reconstructs_covariance(reorder, ragged):
    w, Sig, F = _factor(16, 32, 3, reorder, ragged=ragged)
    P = F.perm
    assert sorted(P.tolist()) == list(range(w.n))
    L = F.dense()
    assert np.abs(L @ L.T - Sig[np.ix_(P, P)]).max() < 50 * w.tol
    assert np.all(np.triu(np.concatenate([np.pad(Bt, ((0, 0), (0, 0))) for Bt in F.B[:1]]), 1) == 0)
    for i, j in F.U:
        assert i > j and F.U[(i, j)].shape[0] == F.tile_off[i + 1] - F.tile_off[i]


def test_tlr_factor_matches_dense_cholesky_at_tight_tolerance():
    w, Sig, F = _factor(16, 64, 5, 2, tol=1e-12)
    P = F.perm
    Ld = np.linalg.cholesky(Sig[np.ix_(P, P)])
    assert np.abs(F.dense() - Ld).max() < 1e-9


def test_reordering_on_independent_variables_is_the_exact_sort():
    # diagonal covariance: univariate conditioning is exact, so both reorderings
    # must order the blocks by their exact log-probability and sort within blocks
    n, m = 48, 8
    rng = np.random.default_rng(3)
    sd = rng.uniform(0.5, 2.0, n)
    a = np.full(n, -np.inf)
    b = rng.uniform(-1, 1.5, n)
    Sig = np.diag(sd**2)
    geo = np.arange(n)
    sizes = [m] * (n // m)
    q = stats.norm.logcdf(b / sd)
    block_p = q.reshape(-1, m).sum(1)
    want_blocks = np.argsort(block_p, kind="stable")
    for reorder in (1, 2):
        F = factor.tlr_factor(Sig, geo, sizes, a, b, 1e-10, m, reorder)
        got_blocks = [int(F.perm[t * m] // m) for t in range(n // m)]
        assert got_blocks == want_blocks.tolist()
        for t in range(n // m):
            seg = F.perm[t * m:(t + 1) * m]
            assert np.all(np.diff(q[seg]) >= 0)
        assert all(F.rank(i, j) == 0 for (i, j) in F.U)


def test_rbodr_differs_from_bodr_on_correlated_problem():
    # the iterative scheme conditions on earlier blocks, so on a correlated
    # problem its block order is generally not the one-shot order
    w, Sig, F1 = _factor(16, 32, 12, 1)
    _, _, F2 = _factor(16, 32, 12, 2)
    assert sorted(F1.perm.tolist()) == sorted(F2.perm.tolist())
    assert not np.array_equal(F1.perm, F2.perm)


def test_rbodr_with_unit_tiles_is_univariate_conditioning():
    # with tiles of one variable, Algorithm 5 is exactly the univariate
    # reordering of the whole matrix (Trinh & Genz), pinned above by hand
    xy = synth.jittered_grid(5, 31)
    Sig = geometry.covariance(xy, 0, (0.3,), 1e-8)
    a, b = synth.limits_uniform(25, 32)
    b = b - 0.5
    F = factor.tlr_factor(Sig, np.arange(25), [1] * 25, a, b, 1e-12, 1, 2)
    uc = factor.univariate_conditioning(Sig, a, b)
    assert np.array_equal(F.perm, uc.order)
    assert np.allclose([Bt[0, 0] for Bt in F.B], np.diag(uc.L), rtol=1e-12)


def test_within_tile_reordering_keeps_the_covariance_and_lowers_the_error():
    # the reordered factor is a factor of the permuted covariance (to the truncation
    # error), keeps every off-diagonal rank, estimates the same probability, and at
    # equal N its QMC error is smaller than the geometric order's on fresh limits
    import math
    from oracle import sov
    w = synth.small_workload(24, 64, 90, n_shifts=10, n_points=500, tol=1e-8)
    perm0, sizes = geometry.kd_order(w.xy, w.m)
    Sig = geometry.covariance(w.xy, w.kernel, w.params, w.nugget)
    F0 = factor.tlr_factor(Sig, perm0, sizes, w.a, w.b, w.tol, w.m, factor.REORDER_NONE)
    L0 = F0.dense()
    for seed, mu, sd in ((3, 2.5, 1.0), (5, 2.0, 0.8)):
        rng = np.random.default_rng(seed)
        b2 = rng.normal(mu, sd, w.n)
        a2 = np.full(w.n, -np.inf)
        F1 = factor.reorder_within_tiles(F0, a2, b2)
        L1 = F1.dense()
        assert np.abs(L1 @ L1.T - Sig[np.ix_(F1.perm, F1.perm)]).max() < 50 * w.tol
        # the same factor up to the permutation and the orthogonal rotation: L L^T exactly
        inv = np.argsort(F1.perm)
        P = np.argsort(F0.perm)
        assert np.abs((L1 @ L1.T)[np.ix_(inv[F0.perm], inv[F0.perm])] - L0 @ L0.T).max() < 1e-12
        assert all(F1.U[k].shape == F0.U[k].shape for k in F0.U)
        assert all(np.all(np.diag(B) > 0) and np.allclose(np.triu(B, 1), 0) for B in F1.B)
        # within each tile only a permutation of the same variables
        for t in range(F0.r):
            o = F0.tile_off
            assert sorted(F1.perm[o[t]:o[t + 1]].tolist()) == sorted(F0.perm[o[t]:o[t + 1]].tolist())
        sh = synth.lattice_shifts(10, w.n + 1, seed)
        r0 = sov.solve(F0, a2, b2, math.inf, sh, 500)
        r1 = sov.solve(F1, a2, b2, math.inf, sh, 500)
        assert abs(r0["logp"] - r1["logp"]) <= 3 * math.hypot(r0["err"], r1["err"])
        assert r1["err"] < r0["err"]


# ---- the TLR-arithmetic factor (covariance compressed first, truncated products) ----

def _factor_truncated(n_side, m, seed, reorder, tol, ragged=None, max_rank=None, nugget=None):
    w = synth.small_workload(n_side, m, seed, ragged_n=ragged, tol=tol)
    perm0, sizes = geometry.kd_order(w.xy, w.m)
    Sig = geometry.covariance(w.xy, w.kernel, w.params, w.nugget if nugget is None else nugget)
    cap = w.m if max_rank is None else max_rank
    F = factor.tlr_factor_truncated(Sig, perm0, sizes, w.a, w.b, tol, cap, reorder)
    return w, Sig, perm0, sizes, F


@pytest.mark.parametrize("reorder", [0, 1, 2])
def test_truncated_factor_is_the_cholesky_factor_at_tight_tolerance(reorder):
    # with nothing truncated away, the TLR arithmetic is exact: the factor is
    # NumPy's Cholesky factor of the permuted covariance, and the order is the
    # one of the exact-Schur factorisation (same decisions on the same blocks)
    w, Sig, perm0, sizes, F = _factor_truncated(12, 24, 41, reorder, 1e-13, ragged=130)
    P = F.perm
    assert sorted(P.tolist()) == list(range(w.n))
    Ld = np.linalg.cholesky(Sig[np.ix_(P, P)])
    assert np.abs(F.dense() - Ld).max() < 1e-9
    E = factor.tlr_factor(Sig, perm0, sizes, w.a, w.b, 1e-13, w.m, reorder)
    assert np.array_equal(P, E.perm)


@pytest.mark.parametrize("reorder", [0, 2])
def test_truncated_factor_error_follows_the_tolerance(reorder):
    # every truncation leaves at most tol per entry; the reconstruction error
    # of L L^T grows with tol (a few tol per tile along the update chain) and
    # vanishes at tight tol; ranks never exceed the cap
    errs = []
    for tol in (1e-3, 1e-5, 1e-9):
        w, Sig, _, _, F = _factor_truncated(16, 32, 42, reorder, tol)
        L = F.dense()
        e = np.abs(L @ L.T - Sig[np.ix_(F.perm, F.perm)]).max()
        assert e <= 4 * F.r * tol, (tol, e)
        assert all(F.rank(i, j) <= w.m for (i, j) in F.U)
        errs.append(e)
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] > 1e-5


def test_truncated_factor_close_to_exact_schur_factor():
    # without reordering both arithmetics factor the same matrix in the same
    # order: their factors differ by the truncation of the Schur tiles only
    for tol in (1e-4, 1e-7):
        w, Sig, perm0, sizes, F = _factor_truncated(16, 32, 43, 0, tol)
        E = factor.tlr_factor(Sig, perm0, sizes, w.a, w.b, tol, w.m, 0)
        assert np.array_equal(F.perm, E.perm)
        d = np.abs(F.dense() - E.dense()).max()
        assert d <= 4 * F.r * tol, (tol, d)


def test_truncated_factor_rank_cap_counts_capped_truncations():
    w, Sig, _, _, F = _factor_truncated(12, 36, 44, 2, 1e-10, max_rank=2)
    assert F.capped_tiles > 0
    assert all(F.rank(i, j) <= 2 for (i, j) in F.U)


def test_truncated_rbodr_with_unit_tiles_is_univariate_conditioning():
    xy = synth.jittered_grid(5, 31)
    Sig = geometry.covariance(xy, 0, (0.3,), 1e-8)
    a, b = synth.limits_uniform(25, 32)
    b = b - 0.5
    F = factor.tlr_factor_truncated(Sig, np.arange(25), [1] * 25, a, b, 1e-13, 1, 2)
    uc = factor.univariate_conditioning(Sig, a, b)
    assert np.array_equal(F.perm, uc.order)
    assert np.allclose([Bt[0, 0] for Bt in F.B], np.diag(uc.L), rtol=1e-10)


def test_truncated_reordering_on_independent_variables_is_the_exact_sort():
    n, m = 48, 8
    rng = np.random.default_rng(3)
    sd = rng.uniform(0.5, 2.0, n)
    a = np.full(n, -np.inf)
    b = rng.uniform(-1, 1.5, n)
    q = stats.norm.logcdf(b / sd)
    want_blocks = np.argsort(q.reshape(-1, m).sum(1), kind="stable")
    for reorder in (1, 2):
        F = factor.tlr_factor_truncated(np.diag(sd**2), np.arange(n), [m] * (n // m), a, b, 1e-10, m, reorder)
        assert [int(F.perm[t * m] // m) for t in range(n // m)] == want_blocks.tolist()
        for t in range(n // m):
            assert np.all(np.diff(q[F.perm[t * m:(t + 1) * m]]) >= 0)
        assert all(F.rank(i, j) == 0 for (i, j) in F.U)
