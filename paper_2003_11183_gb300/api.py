"""Python binding of libtlrmvn (include/tlrmvn.h): the same entry points, with
numpy arrays for host data and torch CUDA tensors for device data.  This
module only marshals arguments; every step of the computation runs in the
library's CUDA kernels.  It raises TlrmvnError on any non-zero status.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np

from . import _lib as L

FP64, FP32, BF16_SHIFT, FP16_SHIFT = 0, 1, 2, 3
REORDER_NONE, REORDER_BLOCK, REORDER_ITERATIVE = 0, 1, 2
SCHUR_EXACT, SCHUR_TLR = 0, 1
KERNEL_EXP, KERNEL_MATERN15, KERNEL_EXP_MATERN15 = 0, 1, 2
E_INVAL, E_NOT_SPD, E_NOMEM, E_CUDA, E_FORMAT, E_NOTSUP, E_TIMEOUT, E_RANK, E_BUSY = 1, 2, 3, 4, 5, 6, 7, 8, 9


class TlrmvnError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = L.load()
        self.status = status
        super().__init__(f"{where}: {lib.tlrmvn_strerror(status).decode()} ({lib.tlrmvn_last_error().decode()})")


def _check(status: int, where: str):
    if status != 0:
        raise TlrmvnError(status, where)


def _dp(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(L.c_double_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Factor:
    """Owns a tlrmvn_factor_t; freed by close() or garbage collection."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def close(self):
        if self.handle and self.handle.value:
            L.load().tlrmvn_factor_free(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _fopts(tile: int, tol: float, max_rank: int, reorder: int, stream, strict_rank: bool = False,
           schur: int = 0) -> L.FactorOpts:
    return L.FactorOpts(int(tile), float(tol), int(max_rank), int(reorder), _stream_ptr(stream),
                        1 if strict_rank else 0, int(schur))


def tlrmvn_factor_kernel(xy, kernel: int, params, nugget: float, a_ref, b_ref, tile: int, tol: float,
                         max_rank: int = 0, reorder: int = REORDER_ITERATIVE, stream=None,
                         strict_rank: bool = False, schur: int = 0) -> Factor:
    lib = L.load()
    xy = _f64(xy).reshape(-1, 2)
    p = _f64(list(params) + [0.0] * (2 - len(params)))
    a = None if a_ref is None else _f64(a_ref)
    b = None if b_ref is None else _f64(b_ref)
    out = C.c_void_p()
    o = _fopts(tile, tol, max_rank, reorder, stream, strict_rank, schur)
    _check(lib.tlrmvn_factor_kernel(_dp(xy), xy.shape[0], int(kernel), _dp(p), float(nugget), _dp(a), _dp(b),
                                    C.byref(o), C.byref(out)), "tlrmvn_factor_kernel")
    return Factor(out.value)


def tlrmvn_factor_dense(cov, a_ref, b_ref, tile: int, tol: float, max_rank: int = 0,
                        reorder: int = REORDER_ITERATIVE, stream=None, strict_rank: bool = False,
                        schur: int = 0) -> Factor:
    lib = L.load()
    cov = np.asfortranarray(cov, dtype=np.float64)
    n = cov.shape[0]
    a = None if a_ref is None else _f64(a_ref)
    b = None if b_ref is None else _f64(b_ref)
    out = C.c_void_p()
    o = _fopts(tile, tol, max_rank, reorder, stream, strict_rank, schur)
    _check(lib.tlrmvn_factor_dense(cov.ctypes.data_as(L.c_double_p), n, n, _dp(a), _dp(b), C.byref(o), C.byref(out)),
           "tlrmvn_factor_dense")
    return Factor(out.value)


def tlrmvn_factor_reorder_tiles(f: Factor, a, b, stream=None) -> Factor:
    """A new factor of the same covariance with every tile's variables reordered for
    the limits (a, b) (original order); see tlrmvn_factor_reorder_tiles."""
    a = _f64(a)
    b = _f64(b)
    out = C.c_void_p()
    _check(L.load().tlrmvn_factor_reorder_tiles(f.handle, _dp(a), _dp(b), _stream_ptr(stream), C.byref(out)),
           "tlrmvn_factor_reorder_tiles")
    return Factor(out.value)


def tlrmvn_factor_info(f: Factor) -> dict:
    lib = L.load()
    n, k = C.c_int64(), C.c_int64()
    r, m, cp = C.c_int(), C.c_int(), C.c_int()
    _check(lib.tlrmvn_factor_info(f.handle, C.byref(n), C.byref(r), C.byref(m), C.byref(k), C.byref(cp)),
           "tlrmvn_factor_info")
    return {"n": n.value, "r": r.value, "m": m.value, "k_total": k.value, "capped": cp.value}


def tlrmvn_factor_ranks(f: Factor) -> np.ndarray:
    """(r, r) int32 ranks of the off-diagonal tiles, rank[i, j] for i > j."""
    lib = L.load()
    r = tlrmvn_factor_info(f)["r"]
    out = np.zeros(r * r, dtype=np.int32)
    _check(lib.tlrmvn_factor_ranks(f.handle, out.ctypes.data_as(C.POINTER(C.c_int32))), "tlrmvn_factor_ranks")
    return out.reshape(r, r)


def tlrmvn_factor_export(f: Factor) -> bytes:
    lib = L.load()
    nb = C.c_size_t(0)
    _check(lib.tlrmvn_factor_export(f.handle, None, C.byref(nb)), "tlrmvn_factor_export")
    buf = C.create_string_buffer(nb.value)
    _check(lib.tlrmvn_factor_export(f.handle, buf, C.byref(nb)), "tlrmvn_factor_export")
    return buf.raw[:nb.value]


def tlrmvn_factor_import(buf: bytes) -> Factor:
    lib = L.load()
    out = C.c_void_p()
    cbuf = C.create_string_buffer(bytes(buf), len(buf))
    _check(lib.tlrmvn_factor_import(cbuf, len(buf), C.byref(out)), "tlrmvn_factor_import")
    return Factor(out.value)


class BatchPlan:
    """tlrmvn_batch_t: many factors solved by one persistent launch (replayed CUDA graph)."""

    def __init__(self, factors, nu, n_shifts: int, n_points: int, seed: int = 0, periodize: bool = True,
                 precision: int = FP32):
        lib = L.load()
        self.factors = list(factors)  # keep the handles alive
        self.sizes = [tlrmvn_factor_info(f)["n"] for f in self.factors]
        count = len(self.factors)
        hs = (C.c_void_p * count)(*[f.handle.value for f in self.factors])
        nus = _f64(nu if np.ndim(nu) else [nu] * count)
        o, _ = _opts(precision, n_shifts, n_points, periodize, None, seed, 0, None, 0)
        out = C.c_void_p()
        _check(lib.tlrmvn_batch_create(count, hs, _dp(nus), C.byref(o), C.byref(out)), "tlrmvn_batch_create")
        self.handle = out
        self.count = count

    def run(self, a_list, b_list):
        """Returns (logp, err) arrays of length count."""
        lib = L.load()
        a_arr = [_f64(a) for a in a_list]
        b_arr = [_f64(b) for b in b_list]
        pa = (L.c_double_p * self.count)(*[_dp(x) for x in a_arr])
        pb = (L.c_double_p * self.count)(*[_dp(x) for x in b_arr])
        lp = np.empty(self.count)
        er = np.empty(self.count)
        _check(lib.tlrmvn_batch_run(self.handle, pa, pb, _dp(lp), _dp(er)), "tlrmvn_batch_run")
        return lp, er

    def tune(self, a_list, b_list, cache_path: str | None = None, force: bool = False) -> dict:
        """Autotune the persistent grid on these limits (tlrmvn_batch_tune); returns the choice."""
        a_arr = [_f64(a) for a in a_list]
        b_arr = [_f64(b) for b in b_list]
        pa = (L.c_double_p * self.count)(*[_dp(x) for x in a_arr])
        pb = (L.c_double_p * self.count)(*[_dp(x) for x in b_arr])
        k, ms = C.c_int(), C.c_double()
        cp = None if cache_path is None else str(cache_path).encode()
        _check(L.load().tlrmvn_batch_tune(self.handle, pa, pb, cp, 1 if force else 0, C.byref(k), C.byref(ms)),
               "tlrmvn_batch_tune")
        return {"ctas_per_sm": k.value, "ms": ms.value}

    def close(self):
        if self.handle and self.handle.value:
            L.load().tlrmvn_batch_free(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tlrmvn_prob_batch(factors, a_list, b_list, nu, n_shifts: int, n_points: int, seed: int = 0,
                      periodize: bool = True, precision: int = FP32):
    """One-shot batched solve: (logp, err) arrays."""
    plan = BatchPlan(factors, nu, n_shifts, n_points, seed, periodize, precision)
    try:
        return plan.run(a_list, b_list)
    finally:
        plan.close()


def tlrmvn_prob_scratch_bytes(f: Factor, precision: int = FP32, n_shifts: int = 10, n_points: int = 1000,
                              sample_chunk: int = 0) -> int:
    """Device scratch bytes of one request with these options on factor f."""
    n = tlrmvn_factor_info(f)["n"]
    o, _ = _opts(precision, n_shifts, n_points, True, None, 0, sample_chunk, None, n)
    nb = C.c_int64()
    _check(L.load().tlrmvn_prob_scratch_bytes(f.handle, C.byref(o), C.byref(nb)), "tlrmvn_prob_scratch_bytes")
    return nb.value


class Server:
    """tlrmvn_server_t: resident factors, requests admitted as lanes and memory free up."""

    def __init__(self, factors, lanes: int = 4, memory_budget: int = 16 << 30):
        lib = L.load()
        self.factors = list(factors)
        self.sizes = [tlrmvn_factor_info(f)["n"] for f in self.factors]
        hs = (C.c_void_p * len(self.factors))(*[f.handle.value for f in self.factors])
        out = C.c_void_p()
        _check(lib.tlrmvn_server_create(hs, len(self.factors), int(lanes), int(memory_budget), C.byref(out)),
               "tlrmvn_server_create")
        self.handle = out

    def submit(self, factor: int, a, b, nu: float = math.inf, precision: int = FP32, n_shifts: int = 10,
               n_points: int = 1000, shifts=None, seed: int = 0, periodize: bool = True, sample_chunk: int = 0) -> int:
        a = _f64(a)
        b = _f64(b)
        n = self.sizes[factor] if 0 <= factor < len(self.sizes) else 0  # the library rejects a bad index
        o, keep = _opts(precision, n_shifts, n_points, periodize, shifts, seed, sample_chunk, None, n)
        rid = C.c_int64()
        _check(L.load().tlrmvn_server_submit(self.handle, int(factor), _dp(a), _dp(b), float(nu), C.byref(o),
                                             C.byref(rid)), "tlrmvn_server_submit")
        del keep
        return rid.value

    def wait(self, rid: int):
        """(logp, err, latency_ms) of a submitted request."""
        lp, er, lat = C.c_double(), C.c_double(), C.c_double()
        _check(L.load().tlrmvn_server_wait(self.handle, int(rid), C.byref(lp), C.byref(er), C.byref(lat)),
               "tlrmvn_server_wait")
        return lp.value, er.value, lat.value

    def stats(self) -> dict:
        st = L.ServerStats()
        _check(L.load().tlrmvn_server_stats(self.handle, C.byref(st)), "tlrmvn_server_stats")
        return {k: getattr(st, k) for k, _ in L.ServerStats._fields_}

    def close(self):
        if self.handle and self.handle.value:
            L.load().tlrmvn_server_free(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tuning_dict(t) -> dict:
    return {"sub": t.sub, "threads": t.threads, "chunk": t.chunk, "tc_ctas": t.tc_ctas, "spt": t.spt,
            "ms": t.ms, "candidates": t.candidates}


def tlrmvn_autotune(f: Factor, a, b, nu: float = math.inf, precision: int = FP32, n_shifts: int = 20,
                    n_points: int = 1000, shifts=None, seed: int = 0, periodize: bool = True,
                    cache_path: str | None = None, force: bool = False, stream=None) -> dict:
    """Times the candidate launch choices for this problem and keeps the fastest on
    the factor (see tlrmvn_autotune in include/tlrmvn.h).  Returns the choice."""
    a = _f64(a)
    b = _f64(b)
    o, keep = _opts(precision, n_shifts, n_points, periodize, shifts, seed, 0, stream, a.size)
    t = L.Tuning()
    cp = None if cache_path is None else str(cache_path).encode()
    _check(L.load().tlrmvn_autotune(f.handle, _dp(a), _dp(b), float(nu), C.byref(o), cp, 1 if force else 0,
                                    C.byref(t)), "tlrmvn_autotune")
    del keep
    return _tuning_dict(t)


def tlrmvn_get_tuning(f: Factor, precision: int) -> dict:
    t = L.Tuning()
    _check(L.load().tlrmvn_get_tuning(f.handle, int(precision), C.byref(t)), "tlrmvn_get_tuning")
    return _tuning_dict(t)


def tlrmvn_set_tuning(f: Factor, precision: int, sub: int = 64, threads: int = 0, chunk: int = 0, tc_ctas: int = 6,
                      spt: int = 1):
    t = L.Tuning(int(sub), int(threads), int(chunk), int(tc_ctas), -1.0, 0, int(spt))
    _check(L.load().tlrmvn_set_tuning(f.handle, int(precision), C.byref(t)), "tlrmvn_set_tuning")


def tlrmvn_estimate_pooled(per_shift_logs) -> tuple[float, float]:
    """(log p_hat, err) of Section 2.1 from per-shift log means gathered on the host
    (computed by the library, float64 on the host; no device work)."""
    ell = _f64(per_shift_logs).ravel()
    lp, er = C.c_double(), C.c_double()
    _check(L.load().tlrmvn_estimate_pooled(_dp(ell), int(ell.size), C.byref(lp), C.byref(er)),
           "tlrmvn_estimate_pooled")
    return lp.value, er.value


NOALLOC_MAX_SHIFTS = 65536


def tlrmvn_estimate_noalloc(per_sample, n_shifts: int, n_points: int, out, per_shift=None, stream=None):
    """Estimator from device per-sample logs without any device allocation.

    per_sample: float64 CUDA tensor (n_shifts * n_points); out: float64 CUDA
    tensor of 2 elements receiving (log p_hat, err); per_shift: optional tensor.
    """
    _check(L.load().tlrmvn_estimate_noalloc(per_sample.data_ptr(), int(n_shifts), int(n_points), out.data_ptr(),
                                            None if per_shift is None else per_shift.data_ptr(),
                                            _stream_ptr(stream)), "tlrmvn_estimate_noalloc")


KC_SHIFT, KC_DIAG, KC_VPROJ, KC_CHI, KC_REDUCE, KC_COUPLE, KC_PREP = 0, 1, 2, 3, 4, 5, 6
KC_NAMES = ("shift", "diag", "vproj", "chi", "reduce", "couple", "prep")


def tlrmvn_profile_enable(on: bool):
    L.load().tlrmvn_profile_enable(1 if on else 0)


def tlrmvn_profile_reset():
    L.load().tlrmvn_profile_reset()


def tlrmvn_profile_get(kernel_class: int):
    """(total device milliseconds, launches) accumulated for one kernel class."""
    ms, n = C.c_double(), C.c_int64()
    _check(L.load().tlrmvn_profile_get(int(kernel_class), C.byref(ms), C.byref(n)), "tlrmvn_profile_get")
    return ms.value, n.value


def tlrmvn_factor_free(f: Factor):
    f.close()


@dataclass
class ExportedFactor:
    """The serialised layout of tlrmvn_factor_export as numpy arrays."""
    n: int
    r: int
    m: int
    tile_off: np.ndarray
    perm: np.ndarray
    rank: np.ndarray      # r x r
    B: np.ndarray         # r x m x m
    U: dict               # (i, j) -> m_i x k
    V: dict               # (i, j) -> m_j x k


def parse_export(buf: bytes) -> ExportedFactor:
    if buf[:8] != b"TLRMVN01":
        raise ValueError("not a tlrmvn factor")
    n, r, m, _ = np.frombuffer(buf, dtype=np.int64, count=4, offset=8)
    n, r, m = int(n), int(r), int(m)
    off = 40
    tile_off = np.frombuffer(buf, np.int64, r + 1, off).copy(); off += 8 * (r + 1)
    perm = np.frombuffer(buf, np.int64, n, off).copy(); off += 8 * n
    rank = np.frombuffer(buf, np.int32, r * r, off).reshape(r, r).copy(); off += 4 * r * r
    B = np.frombuffer(buf, np.float64, r * m * m, off).reshape(r, m, m).copy(); off += 8 * r * m * m
    U, V = {}, {}
    for i in range(r):
        for j in range(i):
            k = int(rank[i, j])
            if not k:
                continue
            mi, mj = int(tile_off[i + 1] - tile_off[i]), int(tile_off[j + 1] - tile_off[j])
            U[(i, j)] = np.frombuffer(buf, np.float64, mi * k, off).reshape(mi, k).copy(); off += 8 * mi * k
            V[(i, j)] = np.frombuffer(buf, np.float64, mj * k, off).reshape(mj, k).copy(); off += 8 * mj * k
    return ExportedFactor(n, r, m, tile_off, perm, rank, B, U, V)


def build_export(n: int, m: int, tile_off, perm, B_tiles, U: dict, V: dict) -> bytes:
    """Serialise a factor given as arrays into the tlrmvn_factor_import layout."""
    r = len(tile_off) - 1
    rank = np.zeros((r, r), dtype=np.int32)
    for (i, j), u in U.items():
        rank[i, j] = u.shape[1]
    Bp = np.zeros((r, m, m))
    for t, Bt in enumerate(B_tiles):
        Bp[t, :Bt.shape[0], :Bt.shape[1]] = np.tril(Bt)
    parts = [b"TLRMVN01", np.array([n, r, m, int(rank.sum())], np.int64).tobytes(),
             np.asarray(tile_off, np.int64).tobytes(), np.asarray(perm, np.int64).tobytes(), rank.tobytes(),
             Bp.tobytes()]
    for i in range(r):
        for j in range(i):
            if rank[i, j]:
                parts.append(np.ascontiguousarray(U[(i, j)], np.float64).tobytes())
                parts.append(np.ascontiguousarray(V[(i, j)], np.float64).tobytes())
    return b"".join(parts)


def _opts(precision, n_shifts, n_points, periodize, shifts, seed, sample_chunk, stream, n):
    keep = None
    sp = None
    if shifts is not None:
        keep = np.ascontiguousarray(shifts, dtype=np.uint64)
        if keep.shape != (n_shifts, n + 1):
            raise ValueError(f"shifts must have shape ({n_shifts}, {n + 1})")
        sp = keep.ctypes.data_as(L.c_u64_p)
    o = L.Opts(int(precision), int(n_shifts), int(n_points), 1 if periodize else 0, sp, int(seed) & (2**64 - 1),
               int(sample_chunk), _stream_ptr(stream))
    return o, keep


def tlrmvn_prob(f: Factor, a, b, nu: float = math.inf, precision: int = FP32, n_shifts: int = 20,
                n_points: int = 1000, shifts=None, seed: int = 0, periodize: bool = True, sample_chunk: int = 0,
                per_shift: bool = False, per_sample: bool = False, stream=None):
    """Host-array call: returns (logp, err, per_shift or None, per_sample or None)."""
    lib = L.load()
    a = _f64(a)
    b = _f64(b)
    n = a.size
    o, keep = _opts(precision, n_shifts, n_points, periodize, shifts, seed, sample_chunk, stream, n)
    lp, er = C.c_double(), C.c_double()
    ps = np.empty(n_shifts) if per_shift else None
    pm = np.empty(n_shifts * n_points) if per_sample else None
    _check(lib.tlrmvn_prob(f.handle, _dp(a), _dp(b), float(nu), C.byref(o), C.byref(lp), C.byref(er), _dp(ps), _dp(pm)),
           "tlrmvn_prob")
    del keep
    return lp.value, er.value, ps, pm


def tlrmvn_prob_device(f: Factor, a, b, out, nu: float = math.inf, precision: int = FP32, n_shifts: int = 20,
                       n_points: int = 1000, shifts=None, seed: int = 0, periodize: bool = True,
                       sample_chunk: int = 0, per_shift=None, per_sample=None, stream=None):
    """Device call: a, b float64 CUDA tensors (original order); out a float64 CUDA
    tensor of 2 elements receiving (logp, err); per_shift / per_sample optional tensors."""
    lib = L.load()
    n = a.numel()
    o, keep = _opts(precision, n_shifts, n_points, periodize, shifts, seed, sample_chunk, stream, n)
    ptr = lambda t: None if t is None else t.data_ptr()
    _check(lib.tlrmvn_prob_device(f.handle, a.data_ptr(), b.data_ptr(), float(nu), C.byref(o), out.data_ptr(),
                                  out.data_ptr() + 8, ptr(per_shift), ptr(per_sample)), "tlrmvn_prob_device")
    del keep


def tlrmvn_selftest_wait_timeout(polls: int = 1000, stream=None) -> int:
    """Status of the bounded-wait self-test (TLRMVN_E_TIMEOUT is the expected outcome)."""
    lib = L.load()
    return lib.tlrmvn_selftest_wait_timeout(int(polls), _stream_ptr(stream) if stream is not None else None)


def tlrmvn_selftest_phi_neg(x) -> np.ndarray:
    """The float sweep's Phi(-x) evaluated on the GPU at float32 values x >= 0."""
    lib = L.load()
    xs = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(xs)
    _check(lib.tlrmvn_selftest_phi_neg(xs.ctypes.data_as(C.POINTER(C.c_float)), int(xs.size),
                                       out.ctypes.data_as(C.POINTER(C.c_float))), "tlrmvn_selftest_phi_neg")
    return out


def tlrmvn_selftest_ndtri(p, lp) -> np.ndarray:
    """The float sweep's normal quantile evaluated on the GPU at float32 (p, log p) pairs."""
    lib = L.load()
    ps = np.ascontiguousarray(p, dtype=np.float32)
    lps = np.ascontiguousarray(lp, dtype=np.float32)
    out = np.empty_like(ps)
    fp = C.POINTER(C.c_float)
    _check(lib.tlrmvn_selftest_ndtri(ps.ctypes.data_as(fp), lps.ctypes.data_as(fp), int(ps.size),
                                     out.ctypes.data_as(fp)), "tlrmvn_selftest_ndtri")
    return out


def tlrmvn_measure_fp32_peak(stream=None) -> float:
    """Measured float32 FMA throughput of the current device, TFLOP/s."""
    t = C.c_double()
    _check(L.load().tlrmvn_measure_fp32_peak(_stream_ptr(stream), C.byref(t)), "tlrmvn_measure_fp32_peak")
    return t.value
