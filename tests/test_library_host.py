"""Host-side checks of the CUDA library that need no GPU: it builds for sm_103a,
loads, exports every entry point declared in include/tlrmvn.h, and rejects bad
arguments before touching a device."""
import ctypes as C
import math
import os
import re
import subprocess

import numpy as np
import pytest

import __graft_entry__ as ge

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ge.build()
    from paper_2003_11183_gb300 import _lib
    return _lib.load()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "tlrmvn.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(tlrmvn_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_entry_points():
    fns = header_functions()
    for want in ("tlrmvn_factor_kernel", "tlrmvn_factor_dense", "tlrmvn_prob", "tlrmvn_prob_device",
                 "tlrmvn_factor_export", "tlrmvn_factor_import", "tlrmvn_factor_free", "tlrmvn_strerror"):
        assert want in fns


def test_library_exports_every_declared_symbol(lib):
    from paper_2003_11183_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(tlrmvn_\w+)", out))
    for fn in header_functions():
        assert fn in exported, fn
        assert fn in _lib.SIGNATURES, fn


def test_build_targets_sm103a_only():
    from paper_2003_11183_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(lib):
    assert lib.tlrmvn_strerror(0) == b"ok"
    assert lib.tlrmvn_strerror(1) == b"invalid argument"
    assert lib.tlrmvn_strerror(2).startswith(b"covariance")


def test_bad_arguments_rejected_without_gpu(lib):
    from paper_2003_11183_gb300 import api, _lib
    out = C.c_void_p()
    xy = np.zeros((4, 2))
    p = np.array([0.1, 0.0])
    o = _lib.FactorOpts(0, 1e-8, 0, 0, None)  # tile 0
    assert lib.tlrmvn_factor_kernel(xy.ctypes.data_as(_lib.c_double_p), 4, 0, p.ctypes.data_as(_lib.c_double_p),
                                    0.0, None, None, C.byref(o), C.byref(out)) == api.E_INVAL
    o = _lib.FactorOpts(2, 1e-8, 0, 2, None)  # reordering without limits
    assert lib.tlrmvn_factor_kernel(xy.ctypes.data_as(_lib.c_double_p), 4, 0, p.ctypes.data_as(_lib.c_double_p),
                                    0.0, None, None, C.byref(o), C.byref(out)) == api.E_INVAL
    a = np.array([0.0, 0.0, 0.0, 0.0])
    b = np.array([1.0, -1.0, 1.0, 1.0])  # a_1 > b_1
    assert lib.tlrmvn_factor_kernel(xy.ctypes.data_as(_lib.c_double_p), 4, 0, p.ctypes.data_as(_lib.c_double_p),
                                    0.0, a.ctypes.data_as(_lib.c_double_p), b.ctypes.data_as(_lib.c_double_p),
                                    C.byref(o), C.byref(out)) == api.E_INVAL
    o = _lib.FactorOpts(2, 1e-8, 0, 0, None, 0, 7)  # unknown Schur arithmetic
    assert lib.tlrmvn_factor_kernel(xy.ctypes.data_as(_lib.c_double_p), 4, 0, p.ctypes.data_as(_lib.c_double_p),
                                    0.0, None, None, C.byref(o), C.byref(out)) == api.E_INVAL
    assert b"schur" in lib.tlrmvn_last_error()
    assert lib.tlrmvn_prob(None, None, None, math.inf, None, None, None, None, None) == api.E_INVAL
    assert lib.tlrmvn_factor_import(b"garbage!" * 8, 64, C.byref(out)) == api.E_FORMAT
    assert b"magic" in lib.tlrmvn_last_error()


def test_export_layout_round_trip_on_host():
    # build_export / parse_export agree with each other and with the header's layout
    from paper_2003_11183_gb300.api import build_export, parse_export
    rng = np.random.default_rng(0)
    tile_off = np.array([0, 3, 6, 8])
    B = [np.tril(rng.normal(size=(s, s))) for s in (3, 3, 2)]
    U = {(1, 0): rng.normal(size=(3, 2)), (2, 0): rng.normal(size=(2, 1)), (2, 1): rng.normal(size=(2, 2))}
    V = {(1, 0): rng.normal(size=(3, 2)), (2, 0): rng.normal(size=(3, 1)), (2, 1): rng.normal(size=(3, 2))}
    perm = rng.permutation(8)
    buf = build_export(8, 3, tile_off, perm, B, U, V)
    ex = parse_export(buf)
    assert ex.n == 8 and ex.r == 3 and ex.m == 3
    assert np.array_equal(ex.perm, perm) and np.array_equal(ex.tile_off, tile_off)
    assert ex.rank[1, 0] == 2 and ex.rank[2, 0] == 1 and ex.rank[2, 1] == 2 and ex.rank[0, 1] == 0
    for k in U:
        assert np.array_equal(ex.U[k], U[k]) and np.array_equal(ex.V[k], V[k])
    assert np.array_equal(ex.B[2, :2, :2], B[2]) and ex.B[2, 2, 2] == 0
    assert len(buf) == 40 + 8 * 4 + 8 * 8 + 4 * 9 + 8 * 27 + 8 * (6 + 6 + 2 + 3 + 4 + 6)


def test_pooled_estimate_equals_the_oracle_estimator(lib):
    # Section 2.1 estimate over per-shift log means, by the library on the host,
    # against the oracle's estimator of the same per-sample values
    from oracle import sov
    from paper_2003_11183_gb300 import api
    rng = np.random.default_rng(3)
    for M, N, scale in ((7, 50, 1.0), (2, 10, 30.0), (40, 3, 0.01)):
        logP = rng.normal(-80.0, scale, size=(M, N))
        logp, err, ell = sov.estimate(logP.ravel(), M, N)
        got = api.tlrmvn_estimate_pooled(ell)
        assert abs(got[0] - logp) <= 1e-13 * abs(logp) and abs(got[1] - err) <= 1e-12 * err
    # one shift: no error estimate; shifts of zero probability are kept by the log-sum-exp
    lp, er = api.tlrmvn_estimate_pooled([-3.0])
    assert lp == -3.0 and math.isnan(er)
    lp, er = api.tlrmvn_estimate_pooled([-2.0, -np.inf])
    assert abs(lp - (-2.0 - math.log(2.0))) < 1e-15 and er > 0
    lp, er = api.tlrmvn_estimate_pooled([-np.inf, -np.inf])
    assert lp == -np.inf and math.isnan(er)


def test_pooled_estimate_rejects_bad_values(lib):
    from paper_2003_11183_gb300 import api
    for bad in ([np.nan, -1.0], [np.inf], []):
        with pytest.raises(api.TlrmvnError) as e:
            api.tlrmvn_estimate_pooled(bad)
        assert e.value.status == api.E_INVAL
