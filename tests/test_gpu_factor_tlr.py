"""GPU: the factorisation in tile-low-rank arithmetic (TLRMVN_SCHUR_TLR; Section 3.3,
Algorithm 5 with the covariance compressed by ACA first and every product with
Sigma_jj^-T and every Schur subtraction truncated) against the oracle's
tlr_factor_truncated on the same inputs:

* the order (integer decisions of float64 univariate conditioning) and every
  tile's rank exactly, the factor entries to 1e-7, the count of capped
  truncations exactly, for the three reorderings and a ragged last tile;
* the rank cap: strict_rank fails with E_RANK, otherwise the capped count matches;
* the float64 integrand on the resulting factor equals the oracle's per sample;
* the dense-covariance entry point builds the same factor.
"""
import math

import numpy as np
import pytest

import synth
from oracle import factor as ofactor, geometry, sov
from tests.helpers import to_oracle_factor

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


def oracle_truncated(w, tol, max_rank, reorder):
    perm0, sizes = geometry.kd_order(w.xy, w.m)
    Sig = geometry.covariance(w.xy, w.kernel, w.params, w.nugget)
    return ofactor.tlr_factor_truncated(Sig, perm0, sizes, w.a, w.b, tol, max_rank, reorder), Sig


def ranks(F):
    return {k: F.U[k].shape[1] for k in F.U}


@pytest.mark.parametrize("reorder", [0, 1, 2])
@pytest.mark.parametrize("ragged", [None, 700])
def test_tlr_arithmetic_factor_matches_the_oracle(tl, reorder, ragged):
    w = synth.small_workload(0 if ragged else 24, 64, 50 + reorder, ragged_n=ragged)
    tol = 1e-5
    OF, Sig = oracle_truncated(w, tol, w.m, reorder)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, tol, 0, reorder,
                                schur=tl.SCHUR_TLR)
    ex = tl.parse_export(tl.tlrmvn_factor_export(F))
    assert np.array_equal(ex.perm, OF.perm)
    assert np.array_equal(ex.tile_off, OF.tile_off)
    GF = to_oracle_factor(ex)
    assert ranks(GF) == ranks(OF)
    assert np.abs(GF.dense() - OF.dense()).max() < 1e-7
    assert tl.tlrmvn_factor_info(F)["capped"] == OF.capped_tiles == 0
    L = GF.dense()
    assert np.abs(L @ L.T - Sig[np.ix_(ex.perm, ex.perm)]).max() < 4 * OF.r * tol


def test_tlr_arithmetic_rank_cap(tl):
    w = synth.small_workload(16, 32, 57)
    OF, _ = oracle_truncated(w, 1e-9, 2, 2)
    assert OF.capped_tiles > 0
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, 1e-9, 2, 2, schur=tl.SCHUR_TLR)
    assert tl.tlrmvn_factor_info(F)["capped"] == OF.capped_tiles
    GF = to_oracle_factor(tl.parse_export(tl.tlrmvn_factor_export(F)))
    assert ranks(GF) == ranks(OF)
    assert np.abs(GF.dense() - OF.dense()).max() < 1e-7
    with pytest.raises(tl.TlrmvnError) as e:
        tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, 1e-9, 2, 2, strict_rank=True,
                                schur=tl.SCHUR_TLR)
    assert e.value.status == tl.E_RANK


def test_tlr_arithmetic_factor_integrand_and_dense_entry(tl):
    w = synth.small_workload(20, 50, 58, nu=7.0, n_shifts=4, n_points=256, ragged_n=390)
    tol = 1e-6
    OF, Sig = oracle_truncated(w, tol, w.m, 2)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, tol, 0, 2, schur=tl.SCHUR_TLR)
    ex = tl.parse_export(tl.tlrmvn_factor_export(F))
    assert np.array_equal(ex.perm, OF.perm)
    GF = to_oracle_factor(ex)
    lp, err, ps, pm = tl.tlrmvn_prob(F, w.a, w.b, w.nu, tl.FP64, w.n_shifts, w.n_points, shifts=w.shifts,
                                     per_shift=True, per_sample=True)
    ref = sov.solve(GF, w.a, w.b, w.nu, w.shifts, w.n_points)
    assert np.all(np.abs(pm - ref["per_sample"]) <= 1e-9 * np.abs(ref["per_sample"]))
    # the same covariance handed over densely: tiles are consecutive runs of m of its order
    perm0, _ = geometry.kd_order(w.xy, w.m)
    Sd = Sig[np.ix_(perm0, perm0)]
    runs = [min(w.m, w.n - t) for t in range(0, w.n, w.m)]
    ODd = ofactor.tlr_factor_truncated(Sd, np.arange(w.n), runs, w.a[perm0], w.b[perm0], tol, w.m, 2)
    Fd = tl.tlrmvn_factor_dense(Sd, w.a[perm0], w.b[perm0], w.m, tol, 0, 2, schur=tl.SCHUR_TLR)
    exd = tl.parse_export(tl.tlrmvn_factor_export(Fd))
    assert np.array_equal(exd.perm, ODd.perm)
    assert np.abs(to_oracle_factor(exd).dense() - ODd.dense()).max() < 1e-7


@pytest.mark.parametrize("schur", [0, 1])
@pytest.mark.parametrize("reorder", [1, 2])
def test_large_tiles_match_the_oracle(tl, reorder, schur):
    # tiles of 256: each diagonal block's Cholesky factor runs in four 64-wide panels and its
    # inverse a warp per column; the order, ranks and factor equal the oracle's (both arithmetics)
    w = synth.small_workload(32, 256, 60 + reorder, tol=1e-6)
    perm0, sizes = geometry.kd_order(w.xy, w.m)
    Sig = geometry.covariance(w.xy, w.kernel, w.params, w.nugget)
    if schur:
        OF = ofactor.tlr_factor_truncated(Sig, perm0, sizes, w.a, w.b, w.tol, w.m, reorder)
    else:
        OF = ofactor.tlr_factor(Sig, perm0, sizes, w.a, w.b, w.tol, w.m, reorder)
    F = tl.tlrmvn_factor_kernel(w.xy, w.kernel, w.params, w.nugget, w.a, w.b, w.m, w.tol, 0, reorder, schur=schur)
    ex = tl.parse_export(tl.tlrmvn_factor_export(F))
    assert np.array_equal(ex.perm, OF.perm)
    GF = to_oracle_factor(ex)
    assert ranks(GF) == {k: v for k, v in ranks(OF).items()}
    assert np.abs(GF.dense() - OF.dense()).max() < 1e-7
