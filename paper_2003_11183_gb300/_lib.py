"""ctypes declarations of the C ABI in include/tlrmvn.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

c_double_p = C.POINTER(C.c_double)
c_u64_p = C.POINTER(C.c_uint64)


class FactorOpts(C.Structure):
    _fields_ = [("tile", C.c_int), ("tol", C.c_double), ("max_rank", C.c_int), ("reorder", C.c_int),
                ("stream", C.c_void_p), ("strict_rank", C.c_int), ("schur", C.c_int)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("n_shifts", C.c_int), ("n_points", C.c_int), ("periodize", C.c_int),
                ("shifts", c_u64_p), ("seed", C.c_uint64), ("sample_chunk", C.c_int64), ("stream", C.c_void_p)]


class Tuning(C.Structure):
    _fields_ = [("sub", C.c_int), ("threads", C.c_int), ("chunk", C.c_int64), ("tc_ctas", C.c_int),
                ("ms", C.c_double), ("candidates", C.c_int), ("spt", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("queued", C.c_int64), ("in_flight", C.c_int), ("peak_in_flight", C.c_int),
                ("overlapped", C.c_int64), ("peak_bytes", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double)]


# every exported symbol of include/tlrmvn.h with its argument and result types
SIGNATURES = {
    "tlrmvn_factor_kernel": (C.c_int, [c_double_p, C.c_int64, C.c_int, c_double_p, C.c_double, c_double_p, c_double_p,
                                        C.POINTER(FactorOpts), C.POINTER(C.c_void_p)]),
    "tlrmvn_factor_dense": (C.c_int, [c_double_p, C.c_int64, C.c_int64, c_double_p, c_double_p, C.POINTER(FactorOpts),
                                       C.POINTER(C.c_void_p)]),
    "tlrmvn_factor_reorder_tiles": (C.c_int, [C.c_void_p, c_double_p, c_double_p, C.c_void_p,
                                              C.POINTER(C.c_void_p)]),
    "tlrmvn_factor_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "tlrmvn_factor_ranks": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "tlrmvn_factor_export": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "tlrmvn_factor_import": (C.c_int, [C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]),
    "tlrmvn_factor_free": (C.c_int, [C.c_void_p]),
    "tlrmvn_prob": (C.c_int, [C.c_void_p, c_double_p, c_double_p, C.c_double, C.POINTER(Opts), c_double_p, c_double_p,
                              c_double_p, c_double_p]),
    "tlrmvn_prob_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(Opts), C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p]),
    "tlrmvn_batch_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), c_double_p, C.POINTER(Opts),
                                      C.POINTER(C.c_void_p)]),
    "tlrmvn_batch_run": (C.c_int, [C.c_void_p, C.POINTER(c_double_p), C.POINTER(c_double_p), c_double_p, c_double_p]),
    "tlrmvn_batch_free": (C.c_int, [C.c_void_p]),
    "tlrmvn_batch_tune": (C.c_int, [C.c_void_p, C.POINTER(c_double_p), C.POINTER(c_double_p), C.c_char_p, C.c_int,
                                    C.POINTER(C.c_int), c_double_p]),
    "tlrmvn_prob_batch": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(c_double_p), C.POINTER(c_double_p),
                                    c_double_p, C.POINTER(Opts), c_double_p, c_double_p]),
    "tlrmvn_server_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int64, C.POINTER(C.c_void_p)]),
    "tlrmvn_server_submit": (C.c_int, [C.c_void_p, C.c_int, c_double_p, c_double_p, C.c_double, C.POINTER(Opts),
                                       C.POINTER(C.c_int64)]),
    "tlrmvn_server_wait": (C.c_int, [C.c_void_p, C.c_int64, c_double_p, c_double_p, c_double_p]),
    "tlrmvn_server_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tlrmvn_server_free": (C.c_int, [C.c_void_p]),
    "tlrmvn_prob_scratch_bytes": (C.c_int, [C.c_void_p, C.POINTER(Opts), C.POINTER(C.c_int64)]),
    "tlrmvn_autotune": (C.c_int, [C.c_void_p, c_double_p, c_double_p, C.c_double, C.POINTER(Opts), C.c_char_p,
                                  C.c_int, C.POINTER(Tuning)]),
    "tlrmvn_get_tuning": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Tuning)]),
    "tlrmvn_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Tuning)]),
    "tlrmvn_estimate_pooled": (C.c_int, [c_double_p, C.c_int64, c_double_p, c_double_p]),
    "tlrmvn_estimate_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tlrmvn_profile_enable": (C.c_int, [C.c_int]),
    "tlrmvn_profile_reset": (C.c_int, []),
    "tlrmvn_profile_get": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "tlrmvn_selftest_wait_timeout": (C.c_int, [C.c_int, C.c_void_p]),
    "tlrmvn_selftest_ndtri": (C.c_int, [C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int,
                                        C.POINTER(C.c_float)]),
    "tlrmvn_selftest_phi_neg": (C.c_int, [C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_float)]),
    "tlrmvn_measure_fp32_peak": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "tlrmvn_strerror": (C.c_char_p, [C.c_int]),
    "tlrmvn_last_error": (C.c_char_p, []),
}

_lib = None


def load(path: str | None = None):
    """Load libtlrmvn.so (built in-tree by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2003_11183_gb300.build.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
