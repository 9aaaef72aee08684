"""GPU parity: the CUDA integrand against the oracle, element by element.

Both sides get the same factor (exported by the library or built by the oracle
and imported), the same lattice and the same shifts.  Tolerances (relative, on
per-shift log-probabilities): FP64 1e-9, FP32 1e-4.  Per-sample log integrands
are compared too: FP64 to 1e-9 relative, FP32 to 1e-4 relative plus 1e-3
absolute (float32 accumulation over a few hundred variables).
"""
import math

import numpy as np
import pytest

import synth
from oracle import sov
from tests.helpers import to_oracle_factor, oracle_factor, export_bytes, sampled_reconstruction_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    return tl


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(np.asarray(b)), 1e-300)


def run_both(tl, F_lib, OF, w, precision, nu=None, samples=None, periodize=True):
    nu = w.nu if nu is None else nu
    lp, err, ps, pm = tl.tlrmvn_prob(F_lib, w.a, w.b, nu, precision, w.n_shifts, w.n_points, shifts=w.shifts,
                                     per_shift=True, per_sample=True, periodize=periodize)
    if samples is None:
        ref = sov.solve(OF, w.a, w.b, nu, w.shifts, w.n_points, periodize)
    else:
        ref = sov.solve(OF, w.a, w.b, nu, w.shifts, w.n_points, periodize, samples=samples)
    return (lp, err, ps, pm), ref


@pytest.mark.parametrize("nu", [math.inf, 7.0])
@pytest.mark.parametrize("ragged", [None, 300])
def test_fp64_per_sample_on_imported_oracle_factor(tl, nu, ragged):
    w = synth.small_workload(16, 64, 31, nu=nu, n_shifts=3, n_points=200, ragged_n=ragged)
    OF, _ = oracle_factor(w)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP64)
    assert np.all(rel(pm, ref["per_sample"]) < 1e-9)
    assert np.all(rel(ps, ref["per_shift"]) < 1e-9)
    assert abs(lp - ref["logp"]) < 1e-9 * abs(ref["logp"])
    assert abs(err - ref["err"]) < 1e-6 * ref["err"]


@pytest.mark.parametrize("nu", [math.inf, 3.0])
def test_fp32_on_imported_oracle_factor(tl, nu):
    w = synth.small_workload(16, 64, 32, nu=nu, n_shifts=4, n_points=300)
    OF, _ = oracle_factor(w)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP32)
    assert np.all(rel(ps, ref["per_shift"]) < 1e-4)
    assert np.all(np.abs(pm - ref["per_sample"]) <= 1e-4 * np.abs(ref["per_sample"]) + 1e-3)


@pytest.mark.parametrize("m", [48, 128])
def test_two_sided_and_upper_tail_limits(tl, m):
    # tiles of 128 put the BF16 path on the whole-tile sweep's two-sided variant
    w = synth.small_workload(12, m, 33, n_shifts=3, n_points=128, limits="twosided")
    w.a[::7] = 1.5
    w.b[::7] = np.inf       # upper-tail one-sided intervals
    OF, _ = oracle_factor(w)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP64)
    assert np.all(rel(pm, ref["per_sample"]) < 1e-9)
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP32)
    assert np.all(rel(ps, ref["per_shift"]) < 1e-4)
    for prec in (tl.BF16_SHIFT, tl.FP16_SHIFT):
        (lp, err, ps, pm), ref = run_both(tl, F, OF, w, prec)
        assert np.all(rel(ps, ref["per_shift"]) < 1e-2)
        assert np.all(np.isfinite(pm))


@pytest.mark.parametrize("m", [48, 128])
def test_deep_tail_limits(tl, m):
    # limits whose interval probabilities lie below the float64 range: one-sided
    # lower tails, two-sided intervals in either half, upper tails.  Every
    # per-sample value is finite and FP64 equals the oracle to 1e-9.  Tiles of
    # 128 take the BF16 path through the whole-tile sweep's log-domain code.
    w = synth.small_workload(12, m, 34, n_shifts=2, n_points=128, limits="twosided")
    w.a[:] = -np.inf
    w.b[:] = np.random.default_rng(5).uniform(0.0, 1.0, w.n)
    w.b[0::5] = -45.0
    w.a[1::5], w.b[1::5] = -41.0, -40.0
    w.a[2::5], w.b[2::5] = 40.0, 41.0
    w.a[3::5], w.b[3::5] = 42.0, np.inf
    OF, _ = oracle_factor(w)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP64)
    assert np.all(np.isfinite(ref["per_sample"])) and np.all(np.isfinite(pm))
    assert np.all(rel(pm, ref["per_sample"]) < 1e-9)
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP32)
    assert np.all(np.isfinite(pm))
    assert np.all(rel(ps, ref["per_shift"]) < 1e-4)
    for prec in (tl.BF16_SHIFT, tl.FP16_SHIFT):
        (lp, err, ps, pm), ref = run_both(tl, F, OF, w, prec)
        assert np.all(np.isfinite(pm))
        assert np.all(rel(ps, ref["per_shift"]) < 1e-2)


@pytest.mark.parametrize("nu", [math.inf, 7.0])
def test_without_periodisation(tl, nu):
    # the lattice used as is (no tent map; the paper does not say which, the
    # library defaults to the tent map and offers both): every
    # precision against the oracle run the same way; tiles of 128 and a ragged
    # sample count (4 x 257) on the BF16 path's whole-tile sweep
    w = synth.small_workload(16, 128, 40, nu=nu, n_shifts=4, n_points=257)
    OF, _ = oracle_factor(w)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP64, periodize=False)
    assert np.all(rel(pm, ref["per_sample"]) < 1e-9)
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP32, periodize=False)
    assert np.all(rel(ps, ref["per_shift"]) < 1e-4)
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.BF16_SHIFT, periodize=False)
    assert np.all(rel(ps, ref["per_shift"]) < 1e-2)
    assert abs(lp - ref["logp"]) <= 3 * max(err, ref["err"])


def test_gpu_factor_matches_oracle_factor(tl):
    for reorder in (0, 1, 2):
        w = synth.small_workload(16, 32, 34, n_shifts=2, n_points=64, reorder=reorder)
        OF, Sig = oracle_factor(w)
        F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 0, reorder)
        ex = tl.parse_export(tl.tlrmvn_factor_export(F))
        assert np.array_equal(ex.perm, OF.perm), reorder        # ordering is integer work: exact
        assert np.array_equal(ex.tile_off, OF.tile_off)
        GF = to_oracle_factor(ex)
        assert np.abs(GF.dense() - OF.dense()).max() < 1e-7
        P = ex.perm
        L = GF.dense()
        assert np.abs(L @ L.T - Sig[np.ix_(P, P)]).max() < 50 * w.tol


def test_gpu_factor_parity_fp64_and_fp32(tl):
    w = synth.small_workload(20, 50, 35, nu=7.0, n_shifts=4, n_points=256, ragged_n=390)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 0, 2)
    OF = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F)))
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP64)
    assert np.all(rel(pm, ref["per_sample"]) < 1e-9)
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP32)
    assert np.all(rel(ps, ref["per_shift"]) < 1e-4)


def test_dense_covariance_entry_point(tl):
    from oracle import geometry
    w = synth.small_workload(10, 25, 36, n_shifts=2, n_points=64)
    Sig = geometry.covariance(w.xy, w.kernel, w.params, w.nugget)
    F = tl.tlrmvn_factor_dense(Sig, w.a, w.b, 25, 1e-10, 0, 2)
    ex = tl.parse_export(tl.tlrmvn_factor_export(F))
    L = to_oracle_factor(ex).dense()
    P = ex.perm
    assert np.abs(L @ L.T - Sig[np.ix_(P, P)]).max() < 1e-8
    OF = to_oracle_factor(ex)
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP64)
    assert np.all(rel(pm, ref["per_sample"]) < 1e-9)


def test_closed_forms_on_gpu(tl):
    # n = 1: every sample equals Phi(b) - Phi(a); all-infinite limits give 0
    from scipy import stats
    F = tl.tlrmvn_factor_dense(np.array([[2.25]]), None, None, 1, 0.0, 0, 0)
    for prec in (tl.FP64, tl.FP32):
        lp, err, ps, pm = tl.tlrmvn_prob(F, [-0.4], [1.1], math.inf, prec, 2, 50, seed=3, per_sample=True)
        want = math.log(stats.norm.cdf(1.1 / 1.5) - stats.norm.cdf(-0.4 / 1.5))
        assert np.allclose(pm, want, rtol=1e-12 if prec == tl.FP64 else 1e-6)
    w = synth.small_workload(8, 16, 37, n_shifts=2, n_points=32)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, None, None, 16, 1e-8, 0, 0)
    lp, err, ps, pm = tl.tlrmvn_prob(F, np.full(64, -np.inf), np.full(64, np.inf), math.inf, tl.FP64, 2, 32,
                                     per_sample=True)
    assert np.all(pm == 0.0) and lp == 0.0
    # bivariate orthant
    rho = 0.6
    F = tl.tlrmvn_factor_dense(np.array([[1.0, rho], [rho, 1.0]]), None, None, 2, 0.0, 0, 0)
    lp, err, _, _ = tl.tlrmvn_prob(F, [-np.inf] * 2, [0.0, 0.0], math.inf, tl.FP64, 10, 4000, seed=5)
    want = 0.25 + math.asin(rho) / (2 * math.pi)
    assert abs(math.exp(lp) - want) <= 4 * err * want + 1e-7


def test_error_paths(tl):
    F = tl.tlrmvn_factor_dense(np.eye(4), None, None, 2, 0.0, 0, 0)
    with pytest.raises(tl.TlrmvnError) as e:
        tl.tlrmvn_prob(F, [0.0] * 4, [-1.0] * 4, math.inf, tl.FP64, 2, 10)
    assert e.value.status == tl.E_INVAL
    bad = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(tl.TlrmvnError) as e:
        tl.tlrmvn_factor_dense(bad, None, None, 2, 0.0, 0, 0)
    assert e.value.status == tl.E_NOT_SPD
    lp, err, _, _ = tl.tlrmvn_prob(F, [-np.inf] * 4, [0.0] * 4, math.inf, tl.FP64, 1, 10)
    assert math.isnan(err)


def test_export_import_round_trip(tl):
    w = synth.small_workload(12, 40, 38, n_shifts=2, n_points=64)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 0, 2)
    buf = tl.tlrmvn_factor_export(F)
    F2 = tl.tlrmvn_factor_import(buf)
    assert tl.tlrmvn_factor_export(F2) == buf
    ranks = tl.tlrmvn_factor_ranks(F)
    assert np.array_equal(ranks, tl.parse_export(buf).rank) and ranks.sum() == tl.tlrmvn_factor_info(F)["k_total"]
    r1 = tl.tlrmvn_prob(F, w.a, w.b, math.inf, tl.FP64, 2, 64, shifts=w.shifts)
    r2 = tl.tlrmvn_prob(F2, w.a, w.b, math.inf, tl.FP64, 2, 64, shifts=w.shifts)
    assert r1[0] == r2[0]


def test_config1_full_size_fp64(tl):
    # n = 256, m = 64, tol 1e-8, iterative block reordering, 20 x 500, FP64
    w = synth.workload(1)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, w.max_rank, w.reorder)
    OF = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F)))
    _check_factor(OF, w)
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, tl.FP64)
    assert np.all(rel(ps, ref["per_shift"]) < 1e-9)
    assert np.all(rel(pm, ref["per_sample"]) < 1e-9)
    own, _ = oracle_factor(w)
    assert np.array_equal(own.perm, OF.perm)


@pytest.mark.parametrize("precision", ["BF16_SHIFT", "FP16_SHIFT"])
@pytest.mark.parametrize("nu", [math.inf, 7.0])
@pytest.mark.parametrize("m,ragged,points", [(64, None, 512), (50, 390, 512), (128, 390, 301)])
def test_bf16_shift_path(tl, nu, m, ragged, points, precision):
    # bf16 tensor-core shifts: per-shift log-probability within 1e-2 relative,
    # and the estimate within 3 QMC standard errors of the oracle's.  Tiles of
    # 128 take the whole-tile sweep (two 64-variable sub-tiles, the last tile 6
    # variables), with 8 x 301 samples: a ragged last block of 128.
    w = synth.small_workload(16, m, 39, nu=nu, n_shifts=8, n_points=points, ragged_n=ragged)
    OF, _ = oracle_factor(w)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    (lp, err, ps, pm), ref = run_both(tl, F, OF, w, getattr(tl, precision))
    assert np.all(rel(ps, ref["per_shift"]) < 1e-2)
    assert abs(lp - ref["logp"]) <= 3 * max(err, ref["err"])
    assert np.all(np.isfinite(pm))


@pytest.mark.parametrize("nu,n_shifts,n_points", [(math.inf, 4, 256), (7.0, 4, 256), (math.inf, 3, 301)])
def test_bf16_split_coupling_without_low_rank(tl, nu, n_shifts, n_points):
    # Block-diagonal covariance in tiles of 256 (four 64-variable sub-tiles each)
    # and a ragged last tile of 150: no low-rank blocks, so the BF16-shift path's
    # only reduced precision is the coupling between sub-tiles, on tensor cores
    # with split operands (x = hi + lo in bf16, relative error ~1e-5).  A
    # single-bf16 coupling is off by about 1 in the per-sample log on this
    # strongly correlated (1-D exponential, range 0.3) covariance; the split one
    # stays near float32.
    rng = np.random.default_rng(7)
    sizes = [256, 256, 256, 150]
    n = sum(sizes)
    Sig = np.zeros((n, n))
    o = 0
    for s in sizes:
        x = np.sort(rng.uniform(0.0, 1.0, s))
        Sig[o:o + s, o:o + s] = np.exp(-np.abs(x[:, None] - x[None, :]) / 0.3) + 1e-8 * np.eye(s)
        o += s
    a = np.full(n, -np.inf)
    b = rng.uniform(0.5, 1.5, n)
    F = tl.tlrmvn_factor_dense(Sig, a, b, 256, 1e-8, 0, 0)
    assert tl.tlrmvn_factor_info(F)["k_total"] == 0
    OF = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F)))
    shifts = synth.lattice_shifts(n_shifts, n + 1, 77)
    lp, err, ps, pm = tl.tlrmvn_prob(F, a, b, nu, tl.BF16_SHIFT, n_shifts, n_points, shifts=shifts, per_shift=True,
                                     per_sample=True)
    ref = sov.solve(OF, a, b, nu, shifts, n_points)
    assert np.all(np.abs(pm - ref["per_sample"]) <= 1e-4 * np.abs(ref["per_sample"]) + 5e-2)
    assert np.all(rel(ps, ref["per_shift"]) < 1e-3)


@pytest.fixture(scope="module", params=["grid64", "ragged3900"])
def headline_family(request, tl):
    # A member of the bench workload's family small enough for the oracle: Student-t
    # nu = 7, exponential kernel beta = 0.1, b ~ N(1, 0.5^2), tiles of 512 (eight
    # 64-variable sub-tiles, seven coupling steps each), ACA tolerance 1e-4 with the
    # rank cap 64 binding, Algorithm 4; 8 shifts x 250 points (2,000 samples: 16 CTAs
    # of 128, the last one ragged).  "grid64": 64 x 64 jittered grid, n = 4,096;
    # "ragged3900": 3,900 uniform points, the last tile 316 variables.
    ragged = None if request.param == "grid64" else 3900
    w = synth.small_workload(64, 512, 51, nu=7.0, n_shifts=8, n_points=250, tol=1e-4, max_rank=64,
                             limits="normal", reorder=1, ragged_n=ragged)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, w.max_rank, w.reorder)
    info = tl.tlrmvn_factor_info(F)
    ranks = tl.tlrmvn_factor_ranks(F)
    # the shape this family is meant to exercise: the rank cap binds, some row tile
    # holds more than one 64-deep block of ranks, and every full tile has 8 sub-tiles
    assert info["capped"] > 0 and ranks.max() == 64 and ranks.sum(axis=1).max() > 64 and info["m"] == 512
    OF = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F)))
    ref = sov.solve(OF, w.a, w.b, w.nu, w.shifts, w.n_points)
    return w, F, ref


@pytest.mark.parametrize("precision", ["BF16_SHIFT", "FP16_SHIFT"])
def test_headline_family_bf16_shift_every_sample_and_shift(tl, headline_family, precision):
    # BF16-shift path (the bench's precision) and the FP16-shift path (per-tile
    # scaled fp16 operands) against the oracle on the same factor, every per-sample
    # and every per-shift value: per shift 1e-2 relative, the estimate within 3 QMC
    # standard errors, per sample 1e-2 relative (each sample's log integrand is a sum
    # over thousands of variables whose limit shifts carry 16-bit operand rounding;
    # the derivation is in the design notes)
    w, F, ref = headline_family
    lp, err, ps, pm = tl.tlrmvn_prob(F, w.a, w.b, w.nu, getattr(tl, precision), w.n_shifts, w.n_points,
                                     shifts=w.shifts, per_shift=True, per_sample=True)
    r_shift = rel(ps, ref["per_shift"])
    r_sample = rel(pm, ref["per_sample"])
    assert np.all(np.isfinite(pm))
    assert np.all(r_shift < 1e-2), r_shift.max()
    assert np.all(r_sample < 1e-2), (r_sample.max(), np.median(r_sample))
    assert abs(lp - ref["logp"]) <= 3 * max(err, ref["err"])


def test_headline_family_fp32_every_sample_and_shift(tl, headline_family):
    # FP32 path on the same factor: every per-shift value within 1e-4 relative and
    # every per-sample value within 1e-4 relative of the oracle
    w, F, ref = headline_family
    lp, err, ps, pm = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP32, w.n_shifts, w.n_points, shifts=w.shifts,
                                     per_shift=True, per_sample=True)
    r_shift = rel(ps, ref["per_shift"])
    r_sample = rel(pm, ref["per_sample"])
    assert np.all(r_shift < 1e-4), r_shift.max()
    assert np.all(r_sample < 1e-4), (r_sample.max(), np.median(r_sample))
    assert abs(lp - ref["logp"]) < 1e-4 * abs(ref["logp"])


def _check_factor(OF, w, n_pairs=24, tol_mult=50):
    # every diagonal entry positive and sampled entries of L L^T equal to Sigma
    assert all(np.all(np.diag(Bt) > 0) for Bt in OF.B)
    rng = np.random.default_rng(1)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, w.n, (n_pairs, 2))]
    pairs += [(t, t) for t in rng.integers(0, w.n, 4).tolist()]
    err = sampled_reconstruction_error(OF, w.xy, w.kernel, w.params, w.nugget, pairs)
    assert err < tol_mult * w.tol, err


def _sampled(w, k=6, seed=0):
    rng = np.random.default_rng(seed)
    S = w.n_shifts * w.n_points
    return np.unique(np.concatenate([[0, S - 1], rng.integers(0, S, k)]))


def test_full_size_mvn_n16384_sampled(tl):
    # n = 16,384, exp + Matern kernel, m = 256, tol 1e-5, iterative block
    # reordering, 20 x 5000; FP64 and FP32 per-sample values checked against
    # the oracle on sampled outputs of the same factor
    w = synth.workload(2)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, w.max_rank, w.reorder)
    OF = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F)))
    _check_factor(OF, w)
    sel = _sampled(w)
    ref = sov.solve(OF, w.a, w.b, w.nu, w.shifts, w.n_points, samples=sel)["per_sample"]
    _, _, _, pm64 = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP64, w.n_shifts, w.n_points, shifts=w.shifts,
                                   per_sample=True)
    assert np.all(rel(pm64[sel], ref) < 1e-9)
    lp32, err32, ps32, pm32 = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP32, w.n_shifts, w.n_points, shifts=w.shifts,
                                             per_shift=True, per_sample=True)
    assert np.all(np.abs(pm32[sel] - ref) <= 1e-4 * np.abs(ref) + 1e-2)
    lp64, err64, ps64, _ = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP64, w.n_shifts, w.n_points, shifts=w.shifts,
                                          per_shift=True)
    assert np.all(rel(ps32, ps64) < 1e-4)


def test_full_size_mvt_n65536_sampled(tl):
    # n = 65,536 Student-t (nu = 7), m = 512, tol 1e-4, ranks <= 64, 20 x 5000:
    # the bench's workload.  Sampled per-sample values of the FP32 and BF16-shift
    # paths against the oracle on the same factor; per-shift BF16 within 1e-2 of FP32.
    w = synth.workload(3)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, w.max_rank, w.reorder)
    OF = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F)))
    _check_factor(OF, w)
    sel = _sampled(w, k=4)
    ref = sov.solve(OF, w.a, w.b, w.nu, w.shifts, w.n_points, samples=sel)["per_sample"]
    lp32, err32, ps32, pm32 = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP32, w.n_shifts, w.n_points, shifts=w.shifts,
                                             per_shift=True, per_sample=True)
    assert np.all(rel(pm32[sel], ref) < 1e-4)
    lp16, err16, ps16, pm16 = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.BF16_SHIFT, w.n_shifts, w.n_points,
                                             shifts=w.shifts, per_shift=True, per_sample=True)
    assert np.all(rel(pm16[sel], ref) < 1e-2)
    assert np.all(rel(ps16, ps32) < 1e-2)
    assert abs(lp16 - lp32) <= 3 * err32
    # every per-shift and per-sample value of both reduced precisions against the
    # library's FP64 path (pinned to the oracle at 1e-9 on smaller problems) on the
    # same factor, lattice and shifts, at 20 x 240 points (4,800 samples)
    pts = 240
    kw = dict(shifts=w.shifts, per_shift=True, per_sample=True)
    _, _, ps64, pm64 = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP64, w.n_shifts, pts, **kw)
    sel64 = sel[sel < w.n_shifts * pts]
    ref64 = sov.solve(OF, w.a, w.b, w.nu, w.shifts, pts, samples=sel64)["per_sample"]
    assert np.all(rel(pm64[sel64], ref64) < 1e-9)
    _, _, ps32r, pm32r = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP32, w.n_shifts, pts, **kw)
    _, _, ps16r, pm16r = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.BF16_SHIFT, w.n_shifts, pts, **kw)
    assert np.all(rel(ps32r, ps64) < 1e-4), rel(ps32r, ps64).max()
    assert np.all(rel(pm32r, pm64) < 1e-4), rel(pm32r, pm64).max()
    assert np.all(rel(ps16r, ps64) < 1e-2), rel(ps16r, ps64).max()
    assert np.all(rel(pm16r, pm64) < 1e-2), rel(pm16r, pm64).max()


def test_float_phi_lower_tail_error_bound(tl):
    # the float sweep's Phi(-x) (Mills-ratio fit) against Phi at the same float32
    # inputs in float64: relative error within 1e-6 on [0, 12] (about 8 ulp), and
    # small and non-negative beyond
    from scipy.special import ndtr
    x = np.concatenate([np.linspace(0.0, 12.0, 200001), [12.5, 13.0, 14.0, 20.0, 40.0]]).astype(np.float32)
    got = tl.tlrmvn_selftest_phi_neg(x).astype(np.float64)
    want = ndtr(-x.astype(np.float64))
    inside = x <= 12.0
    assert np.max(np.abs(got[inside] / want[inside] - 1.0)) < 1e-6
    assert np.all(got[~inside] >= 0) and np.all(got[~inside] < 1e-33)


@pytest.mark.parametrize("precision", ["FP64", "FP32", "BF16_SHIFT"])
def test_sample_chunks_change_nothing(tl, precision):
    # a solve in chunks of 768 samples (3 full chunks and a ragged one of 4 x 250
    # samples) gives every sample bit for bit the value of the one-chunk solve:
    # no step mixes samples, and the chunk offset enters only the lattice index
    # (tiles of 128: the BF16 path runs the whole-tile sweep)
    w = synth.small_workload(16, 128, 41, nu=7.0, n_shifts=4, n_points=750)
    OF, _ = oracle_factor(w)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    prec = getattr(tl, precision)
    kw = dict(shifts=w.shifts, per_shift=True, per_sample=True)
    full = tl.tlrmvn_prob(F, w.a, w.b, w.nu, prec, w.n_shifts, w.n_points, **kw)
    part = tl.tlrmvn_prob(F, w.a, w.b, w.nu, prec, w.n_shifts, w.n_points, sample_chunk=768, **kw)
    assert np.array_equal(full[3], part[3])
    assert np.array_equal(full[2], part[2])
    ref = sov.solve(OF, w.a, w.b, w.nu, w.shifts, w.n_points)
    tol = {"FP64": 1e-9, "FP32": 1e-4, "BF16_SHIFT": 1e-2}[precision]
    assert np.all(rel(part[2], ref["per_shift"]) < tol)


def test_rank_cap_policy(tl):
    # a rank cap that binds: by default the capped tiles are counted, with
    # strict_rank the factorisation fails with TLRMVN_E_RANK
    w = synth.small_workload(16, 32, 42, tol=1e-10, max_rank=2)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 2, 1)
    info = tl.tlrmvn_factor_info(F)
    assert info["capped"] > 0 and tl.tlrmvn_factor_ranks(F).max() == 2
    with pytest.raises(tl.TlrmvnError) as e:
        tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 2, 1, strict_rank=True)
    assert e.value.status == tl.E_RANK
    # a cap that does not bind passes under the strict policy
    F2 = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, 1e-4, 0, 1, strict_rank=True)
    assert tl.tlrmvn_factor_info(F2)["capped"] == 0


def test_float_quantile_error_bound(tl):
    # the float sweep's own normal quantile (AS 241, PPND7, evaluated in float32)
    # against the float64 quantile of the same float32 inputs: relative error within
    # 1e-6 (about 8 ulp) on [1e-30, 1/2] and, from the log of the probability alone,
    # down to log p = -700
    from scipy.special import ndtri, ndtri_exp
    p = np.concatenate([np.geomspace(1e-30, 0.5, 200001), np.linspace(0.3, 0.5, 20001)]).astype(np.float32)
    lp = np.log(p.astype(np.float64)).astype(np.float32)
    got = tl.tlrmvn_selftest_ndtri(p, lp).astype(np.float64)
    want = ndtri(p.astype(np.float64))
    ok = want != 0.0
    assert np.max(np.abs(got[ok] / want[ok] - 1.0)) < 1e-6
    assert np.all(got[~ok] == 0.0)
    lpd = -np.geomspace(69.0, 700.0, 20001).astype(np.float32)
    got = tl.tlrmvn_selftest_ndtri(np.zeros_like(lpd), lpd).astype(np.float64)
    want = ndtri_exp(lpd.astype(np.float64))
    assert np.max(np.abs(got / want - 1.0)) < 1e-6


def test_scale_invariance_every_precision(tl):
    # Phi_n(D a, D b; D Sigma D) = Phi_n(a, b; Sigma) (eq. 1): with D = 2^-20 I every
    # step of the path scales exactly, so each per-sample value must be bit for bit
    # that of the unscaled problem in every precision.  The scaled factor's entries
    # (~1e-6) lie below fp16's normal range: the FP16-shift path meets this only
    # through its power-of-two normalisation of the products (global g, per-tile a, c).
    from oracle import geometry
    w = synth.small_workload(20, 128, 44, nu=7.0, n_shifts=4, n_points=300, tol=1e-6)
    Sig = geometry.covariance(w.xy, w.kernel, w.params, w.nugget)
    d = 2.0 ** -20
    F1 = tl.tlrmvn_factor_dense(Sig, w.a, w.b, w.m, w.tol, 0, 1)
    F2 = tl.tlrmvn_factor_dense(Sig * d * d, w.a * d, w.b * d, w.m, w.tol * d, 0, 1)
    e1, e2 = tl.parse_export(tl.tlrmvn_factor_export(F1)), tl.parse_export(tl.tlrmvn_factor_export(F2))
    assert np.array_equal(e1.perm, e2.perm) and np.array_equal(e1.rank, e2.rank)
    assert np.array_equal(e1.B * d, e2.B)
    for prec in (tl.FP64, tl.FP32, tl.BF16_SHIFT, tl.FP16_SHIFT):
        kw = dict(shifts=w.shifts, per_sample=True)
        p1 = tl.tlrmvn_prob(F1, w.a, w.b, w.nu, prec, w.n_shifts, w.n_points, **kw)[3]
        p2 = tl.tlrmvn_prob(F2, w.a * d, w.b * d, w.nu, prec, w.n_shifts, w.n_points, **kw)[3]
        assert np.array_equal(p1, p2), prec
    OF = to_oracle_factor(e1)
    ref = sov.solve(OF, w.a, w.b, w.nu, w.shifts, w.n_points)
    p16 = tl.tlrmvn_prob(F2, w.a * d, w.b * d, w.nu, tl.FP16_SHIFT, w.n_shifts, w.n_points, shifts=w.shifts,
                         per_shift=True)[2]
    assert np.all(rel(p16, ref["per_shift"]) < 1e-2)


@pytest.mark.parametrize("nu", [math.inf, 7.0])
@pytest.mark.parametrize("precision,tol", [("FP64", 1e-9), ("FP32", 1e-4), ("BF16_SHIFT", 1e-2), ("FP16_SHIFT", 1e-2)])
def test_full_size_closed_form_every_sample(tl, precision, tol, nu):
    # n = 65,536, 512-variable tiles, ranks 1..3 (tests.helpers.sources_targets_factor):
    # every per-sample value of 4 x 128 samples against its closed form, computed from
    # the lattice values without the tile recursion (pinned on the oracle at this size
    # by tests/test_oracle_full_size.py)
    from oracle import lattice
    from tests.helpers import closed_form_logf, sources_targets_factor
    n, m, M, N = 65_536, 512, 4, 128
    OF, b = sources_targets_factor(n, m, seed=21)
    F = tl.tlrmvn_factor_import(export_bytes(OF))
    a = np.full(n, -np.inf)
    shifts = synth.lattice_shifts(M, n + 1, 22)
    _, _, _, pm = tl.tlrmvn_prob(F, a, b, nu, getattr(tl, precision), M, N, shifts=shifts, per_sample=True)
    Wall = lattice.qmc_points(lattice.richtmyer_generators(n + 1), shifts, N)
    rs = None
    if math.isfinite(nu):  # Student-t: the sample's scale from lattice coordinate n (SciPy's chi quantile)
        from scipy import stats
        rs = stats.chi.ppf(Wall[:, n], nu) / math.sqrt(nu)
    want = closed_form_logf(OF, b, Wall[:, :n].T, rs)
    assert np.all(np.isfinite(pm))
    assert np.all(rel(pm, want) < tol), rel(pm, want).max()


@pytest.mark.parametrize("precision,tol", [("FP64", 1e-12), ("FP32", 2e-6), ("BF16_SHIFT", 2e-6), ("FP16_SHIFT", 2e-6)])
@pytest.mark.parametrize("one_sided", [True, False])
def test_tiny_and_ragged_problems_every_precision(tl, precision, tol, one_sided):
    # degenerate shapes against closed forms per sample: n = 1 (Phi(b) - Phi(a) with sigma = 1.5;
    # FP64 and FP32, a problem the tensor-core paths are not meant for), and on every path n = 17
    # independent variables in tiles of 16 (a full tile and a one-variable tile; no low-rank
    # blocks), where each sample is the product of the univariate probabilities; one-sided limits
    # take the float paths' one-sided step
    from scipy.special import log_ndtr, ndtr
    prec = getattr(tl, precision)

    def logdiff(a, b):
        a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
        return np.where(np.isneginf(a), log_ndtr(b), np.log(ndtr(b) - ndtr(a)))

    if prec in (tl.FP64, tl.FP32):
        a1 = [-np.inf] if one_sided else [-0.4]
        F = tl.tlrmvn_factor_dense(np.array([[2.25]]), None, None, 1, 0.0, 0, 0)
        _, _, _, pm = tl.tlrmvn_prob(F, a1, [1.1], math.inf, prec, 2, 50, seed=3, per_sample=True)
        want = float(logdiff(np.array(a1) / 1.5, 1.1 / 1.5)[0])
        assert np.allclose(pm, want, rtol=tol, atol=0)
    rng = np.random.default_rng(31)
    n = 17
    b = rng.uniform(0.2, 2.0, n)
    a = np.full(n, -np.inf) if one_sided else b - rng.uniform(0.5, 3.0, n)
    F = tl.tlrmvn_factor_dense(np.eye(n), None, None, 16, 1e-8, 0, 0)
    _, _, _, pm = tl.tlrmvn_prob(F, a, b, math.inf, prec, 3, 40, seed=5, per_sample=True)
    want = float(logdiff(a, b).sum())
    assert np.allclose(pm, want, rtol=tol, atol=0)


@pytest.mark.parametrize("precision", ["FP64", "FP32", "BF16_SHIFT", "FP16_SHIFT"])
def test_degenerate_limits_every_precision(tl, precision):
    # the method's degenerate cases on every path (n = 40 with a real low-rank structure, tiles
    # of 16): limits infinite on both sides give probability 1 (every per-sample log exactly 0);
    # one zero-width interval a_i = b_i gives probability 0 (every per-sample log and the
    # estimate -inf, its error NaN), and the other samples' arithmetic stays finite
    prec = getattr(tl, precision)
    w = synth.small_workload(8, 16, 91, n_shifts=3, n_points=40, ragged_n=40)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, None, None, 16, 1e-6, 0, 0)
    n = len(w.xy)
    lp, err, ps, pm = tl.tlrmvn_prob(F, np.full(n, -np.inf), np.full(n, np.inf), math.inf, prec, 3, 40,
                                     seed=9, per_shift=True, per_sample=True)
    assert np.all(pm == 0.0) and np.all(ps == 0.0) and lp == 0.0
    a = np.full(n, -np.inf)
    b = np.full(n, 1.0)
    a[n // 2] = b[n // 2] = 0.3
    lp, err, ps, pm = tl.tlrmvn_prob(F, a, b, 7.0, prec, 3, 40, seed=9, per_shift=True, per_sample=True)
    assert np.all(np.isneginf(pm)) and np.all(np.isneginf(ps)) and lp == -np.inf and math.isnan(err)
