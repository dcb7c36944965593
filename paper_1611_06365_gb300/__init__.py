"""GB300-native LU factorization with partial pivoting (PA = LU) with
look-ahead, after arXiv:1611.06365 (blocked right-looking LU, section 3;
malleable look-ahead, section 4).

This module is the Python binding of the C ABI in ``include/lu.h``: every
function marshals torch tensors (device memory, streams) into the library's
plain pointers and sizes and calls the entry point of the same name.  All
arithmetic runs in the CUDA kernels of ``liblu.so``; there is no CPU path.

Matrix layout: column-major.  A torch tensor ``T`` of shape (n_cols, ld) that
is contiguous holds the column-major matrix whose column j is ``T[j, :m]``
(``to_colmajor`` / ``from_colmajor`` convert from/to ordinary row-major
matrices).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build_mod

__all__ = [
    "LU_OK", "LU_F64", "LU_F32", "LU_UPDATE_NATIVE", "LU_UPDATE_BF16", "LU_UPDATE_BF16X3", "LU_UPDATE_FP8",
    "LU_UPDATE_F64EMU", "LuError", "lib", "build", "lu_trailing_update_f64", "lu_cholesky", "lu_cholesky_solve",
    "lu_factor", "lu_solve", "lu_solve_noalloc", "lu_solve_noalloc_capacity", "lu_factor_batched", "lu_solve_batched", "lu_solve_mixed",
    "lu_trailing_update", "lu_workspace_size", "lu_status_string", "lu_last_device_status", "lu_get_status",
    "lu_version", "lu_update_timing", "lu_update_timing_read", "lu_trace", "lu_trace_read", "lu_wait_selftest", "lu_div_selftest", "lu_kernel_launches",
    "lu_autotune", "lu_autotune_batched", "lu_tune_get", "lu_tune_put", "lu_tune_save", "lu_tune_load", "lu_tune_count",
    "lu_tune_clear", "lu_plan_info", "lu_peak_probe", "lu_cta_trace", "lu_cta_trace_read", "PROBE_DFMA", "PROBE_FFMA", "PROBE_DMMA", "TUNE_FACTOR", "TUNE_BATCHED", "to_colmajor", "from_colmajor", "MixedReport",
]

LU_F64, LU_F32 = 0, 1
LU_UPDATE_NATIVE, LU_UPDATE_BF16, LU_UPDATE_BF16X3, LU_UPDATE_FP8, LU_UPDATE_F64EMU = 0, 1, 2, 3, 4
LU_OK = 0
LU_ERR_CUDA, LU_ERR_NOMEM, LU_ERR_TIMEOUT, LU_ERR_UNSUPPORTED = -100, -101, -102, -103
LU_ERR_SCRATCH = -104
TUNE_FACTOR, TUNE_BATCHED = 0, 1   # kinds of tuning-table entries
PROBE_DFMA, PROBE_FFMA, PROBE_DMMA = 0, 1, 2   # lu_peak_probe kinds
LU_TRACE_KINDS = ("panel", "swap_left", "ru1", "pf1", "pf2", "ru2")

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


class LuError(RuntimeError):
    def __init__(self, name, code):
        self.code = code
        msg = _lib.lu_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{name} returned {code}: {msg}")


class LuOpts(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("nb_inner", ctypes.c_int), ("panel_ctas", ctypes.c_int),
                ("lookahead", ctypes.c_int), ("update", ctypes.c_int), ("spin_ns", ctypes.c_longlong),
                ("update_ctas", ctypes.c_int), ("sm_share", ctypes.c_int), ("tile", ctypes.c_int),
                ("early_term", ctypes.c_int)]


class TuneResult(ctypes.Structure):
    _fields_ = [("opts", LuOpts), ("ms", ctypes.c_double), ("candidates", ctypes.c_int)]


class MixedOpts(ctypes.Structure):
    _fields_ = [("update", ctypes.c_int), ("nb", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("tol", ctypes.c_double), ("allow_gmres", ctypes.c_int), ("allow_fallback", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("fp64_factor", ctypes.c_int), ("fallback_native", ctypes.c_int),
                ("f32_refactor", ctypes.c_int), ("fallback_ratio", ctypes.c_double)]


class MixedReport(ctypes.Structure):
    _fields_ = [("rung", ctypes.c_int), ("iterations", ctypes.c_int), ("gmres_iters", ctypes.c_int),
                ("fell_back", ctypes.c_int), ("info", ctypes.c_int), ("backward_error", ctypes.c_double),
                ("t_factor_ms", ctypes.c_double), ("t_refine_ms", ctypes.c_double), ("t_total_ms", ctypes.c_double),
                ("forward_error_est", ctypes.c_double), ("f32_refactor", ctypes.c_int), ("cost_stop", ctypes.c_int),
                ("t_fallback_ms", ctypes.c_double), ("cond_est", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile liblu.so for sm_103a (nvcc); returns its path."""
    return _build_mod.build(force=force)


def lib():
    """The loaded liblu.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        path = os.path.join(_HERE, "liblu.so")
        if not os.path.exists(path):
            raise ImportError(f"liblu.so is not built ({path}); run paper_1611_06365_gb300.build()")
        L = ctypes.CDLL(path)
        vp, i, ip = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
        L.lu_factor.argtypes = [i, i, vp, i, ip, ip, ctypes.POINTER(LuOpts), vp]
        L.lu_solve.argtypes = [i, i, i, vp, i, ip, vp, i, vp]
        L.lu_factor_batched.argtypes = [i, i, ip, vp, ip, vp, ip, i, ctypes.POINTER(LuOpts), vp]
        L.lu_solve_batched.argtypes = [i, i, i, ip, vp, ip, vp, vp, ip, i, vp]
        L.lu_solve_mixed.argtypes = [i, i, vp, i, vp, i, vp, i, ctypes.POINTER(MixedOpts),
                                     ctypes.POINTER(MixedReport), vp]
        L.lu_trailing_update.argtypes = [i, i, i, i, vp, i, vp, i, vp, i, vp]
        L.lu_trailing_update_f64.argtypes = [i, i, i, i, vp, i, vp, i, vp, i, vp]
        L.lu_trailing_update_f64.restype = i
        L.lu_cholesky.argtypes = [i, i, vp, i, ip, ctypes.POINTER(LuOpts), vp]
        L.lu_cholesky.restype = i
        L.lu_cholesky_solve.argtypes = [i, i, i, vp, i, vp, i, vp]
        L.lu_cholesky_solve.restype = i
        L.lu_workspace_size.argtypes = [ctypes.c_char_p, i, i, i]
        L.lu_workspace_size.restype = ctypes.c_size_t
        L.lu_status_string.argtypes = [i]
        L.lu_status_string.restype = ctypes.c_char_p
        L.lu_last_device_status.argtypes = [vp, i]
        L.lu_get_status.argtypes = [vp]
        L.lu_get_status.restype = i
        L.lu_version.restype = ctypes.c_char_p
        L.lu_abi_size.argtypes = [ctypes.c_char_p]
        L.lu_abi_size.restype = ctypes.c_size_t
        L.lu_solve_noalloc.argtypes = [i, i, i, vp, i, ip, vp, i, ip, vp]
        L.lu_solve_noalloc.restype = i
        L.lu_solve_noalloc_capacity.restype = ctypes.c_size_t
        L.lu_last_panel_widths.argtypes = [ip, i]
        L.lu_last_panel_widths.restype = i
        L.lu_update_timing.argtypes = [i]
        L.lu_update_timing.restype = i
        L.lu_update_timing_read.argtypes = [ctypes.POINTER(ctypes.c_longlong)] + [ctypes.POINTER(ctypes.c_double)] * 3
        L.lu_update_timing_read.restype = i
        L.lu_kernel_launches.restype = ctypes.c_longlong
        L.lu_div_selftest.argtypes = [i, ctypes.c_longlong, ctypes.c_ulonglong, vp]
        L.lu_div_selftest.restype = ctypes.c_longlong
        L.lu_wait_selftest.argtypes = [ctypes.c_longlong, vp]
        L.lu_wait_selftest.restype = i
        L.lu_trace.argtypes = [i]
        L.lu_trace.restype = i
        L.lu_trace_read.argtypes = [ctypes.POINTER(TraceEvent), i]
        L.lu_trace_read.restype = i
        L.lu_cta_trace.argtypes = [i]
        L.lu_cta_trace.restype = i
        L.lu_cta_trace_read.argtypes = [ctypes.POINTER(CtaEvent), i]
        L.lu_cta_trace_read.restype = i
        L.lu_autotune.argtypes = [i, i, i, ctypes.c_double, ctypes.POINTER(TuneResult), vp]
        L.lu_autotune_batched.argtypes = [i, i, ip, i, ctypes.POINTER(TuneResult), vp]
        L.lu_tune_get.argtypes = [i, i, i, i, ctypes.POINTER(LuOpts)]
        L.lu_tune_put.argtypes = [i, i, i, i, ctypes.POINTER(LuOpts), ctypes.c_double]
        L.lu_tune_save.argtypes = [ctypes.c_char_p]
        L.lu_tune_load.argtypes = [ctypes.c_char_p]
        L.lu_tune_clear.restype = None
        L.lu_peak_probe.argtypes = [i, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), vp]
        L.lu_peak_probe.restype = i
        L.lu_plan_info.argtypes = [i, i, ctypes.POINTER(LuOpts), ctypes.POINTER(LuOpts)]
        L.lu_plan_info.restype = i
        for f in ("lu_autotune", "lu_autotune_batched", "lu_tune_get", "lu_tune_put", "lu_tune_save", "lu_tune_load",
                  "lu_tune_count"):
            getattr(L, f).restype = i
        for f in ("lu_factor", "lu_solve", "lu_factor_batched", "lu_solve_batched", "lu_solve_mixed",
                  "lu_trailing_update", "lu_last_device_status"):
            getattr(L, f).restype = i
        _lib = L
    return _lib


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return LU_F64
    if t.dtype == torch.float32:
        return LU_F32
    raise TypeError(f"unsupported dtype {t.dtype}: float64 or float32")


def _check(name, rc):
    if rc != 0:
        raise LuError(name, rc)
    return rc


def _ld(t):
    """Leading dimension of a column-major (n_cols, ld) tensor.  With a single
    column the stride of dimension 0 is arbitrary in torch (any value is
    contiguous), so the column length is used."""
    if t.dim() != 2:
        return t.shape[0]
    return t.stride(0) if t.shape[0] > 1 else max(t.shape[1], 1)


def _cm_dims(A, n=None):
    """(n, ld) of a column-major tensor of shape (n_cols, ld)."""
    if A.dim() != 2 or (A.stride(1) != 1 and A.shape[1] > 1):
        raise ValueError("column-major matrix expected: a (n_cols, ld) tensor with unit inner stride")
    return (A.shape[0] if n is None else n), _ld(A)


def lu_factor(A, ipiv, info, n=None, *, nb=0, nb_inner=0, panel_ctas=0, lookahead=0,
              update=LU_UPDATE_NATIVE, spin_ns=0, update_ctas=0, sm_share=0, tile=0, early_term=0, stream=None):
    """P A = L U in place (see include/lu.h).  A: column-major (n, lda) tensor."""
    n, lda = _cm_dims(A, n)
    o = LuOpts(nb, nb_inner, panel_ctas, lookahead, update, spin_ns, update_ctas, sm_share, tile, early_term)
    return _check("lu_factor", lib().lu_factor(_dtype_code(A), n, _ptr(A), lda, _ptr(ipiv), _ptr(info),
                                                ctypes.byref(o), _stream(stream)))


def lu_last_panel_widths():
    """Widths of the panels of the last factorization on the current device (a list),
    or None before the first one."""
    cnt = lib().lu_last_panel_widths(None, 0)
    if cnt < 0:
        return None
    buf = (ctypes.c_int * max(cnt, 1))()
    lib().lu_last_panel_widths(buf, cnt)
    return list(buf[:cnt])


def lu_cholesky(A, info, n=None, *, nb=0, lookahead=0, update=LU_UPDATE_NATIVE, spin_ns=0, stream=None):
    """A = L L^T in place (lower triangle) of a symmetric positive definite column-major (n, lda) tensor."""
    n, lda = _cm_dims(A, n)
    o = LuOpts(nb, 0, 0, lookahead, update, spin_ns, 0)
    return _check("lu_cholesky", lib().lu_cholesky(_dtype_code(A), n, _ptr(A), lda, _ptr(info), ctypes.byref(o),
                                                    _stream(stream)))


def lu_cholesky_solve(L, B, n=None, nrhs=None, *, stream=None):
    """B := A^{-1} B with the factor of lu_cholesky.  B: column-major (nrhs, ldb)."""
    n, lda = _cm_dims(L, n)
    nrhs = B.shape[0] if nrhs is None else nrhs
    return _check("lu_cholesky_solve", lib().lu_cholesky_solve(_dtype_code(L), n, nrhs, _ptr(L), lda, _ptr(B), _ld(B),
                                                                _stream(stream)))


def lu_solve(LU, ipiv, B, n=None, nrhs=None, *, stream=None):
    """B := A^{-1} B with the factors of lu_factor.  B: column-major (nrhs, ldb)."""
    n, lda = _cm_dims(LU, n)
    nrhs = B.shape[0] if nrhs is None else nrhs
    ldb = _ld(B)
    return _check("lu_solve", lib().lu_solve(_dtype_code(LU), n, nrhs, _ptr(LU), lda, _ptr(ipiv), _ptr(B), ldb,
                                              _stream(stream)))


def lu_solve_noalloc(LU, ipiv, B, n=None, nrhs=None, *, status=None, stream=None):
    """lu_solve without any memory allocation: the workspace is a fixed array of
    lu_solve_noalloc_capacity() bytes in device memory.  For callers that may
    not allocate during a solve (device memory reserved by another pool,
    latency-critical loops).  Calls that overlap on the GPU must not share it."""
    n, lda = _cm_dims(LU, n)
    nrhs = B.shape[0] if nrhs is None else nrhs
    ldb = _ld(B)
    return _check("lu_solve_noalloc", lib().lu_solve_noalloc(_dtype_code(LU), n, nrhs, _ptr(LU), lda, _ptr(ipiv),
                                                              _ptr(B), ldb, _ptr(status), _stream(stream)))


def lu_solve_noalloc_capacity() -> int:
    return lib().lu_solve_noalloc_capacity()


def lu_factor_batched(dtype_code, ns, A_ptrs, ldas, ipiv_ptrs, infos, max_n, *, nb=0, stream=None):
    """Batched factorization; all arguments are device tensors (pointer arrays as int64).
    nb: 0 automatic, 16 or 32 blocked panel width, 1 the unblocked kernel."""
    o = LuOpts(nb, 0, 0, 0, 0, 0)
    return _check("lu_factor_batched", lib().lu_factor_batched(dtype_code, ns.shape[0], _ptr(ns), _ptr(A_ptrs), _ptr(ldas),
                                                                _ptr(ipiv_ptrs), _ptr(infos), max_n, ctypes.byref(o),
                                                                _stream(stream)))


def lu_solve_batched(dtype_code, nrhs, ns, LU_ptrs, ldas, ipiv_ptrs, B_ptrs, ldbs, max_n, *, stream=None):
    return _check("lu_solve_batched", lib().lu_solve_batched(dtype_code, ns.shape[0], nrhs, _ptr(ns), _ptr(LU_ptrs),
                                                              _ptr(ldas), _ptr(ipiv_ptrs), _ptr(B_ptrs), _ptr(ldbs),
                                                              max_n, _stream(stream)))


def lu_solve_mixed(A, B, X, n=None, *, update=LU_UPDATE_BF16X3, nb=0, max_iter=0, tol=0.0, allow_gmres=1,
                   allow_fallback=1, gmres_restart=0, fp64_factor=0, fallback_native=0, f32_refactor=0,
                   fallback_ratio=0.0, stream=None):
    """Mixed-precision solve A X = B (FP64 in/out).  Returns a MixedReport."""
    n, lda = _cm_dims(A, n)
    nrhs = B.shape[0]
    o = MixedOpts(update, nb, max_iter, tol, allow_gmres, allow_fallback, gmres_restart, fp64_factor, fallback_native,
                  f32_refactor, fallback_ratio)
    rep = MixedReport()
    _check("lu_solve_mixed", lib().lu_solve_mixed(n, nrhs, _ptr(A), lda, _ptr(B), _ld(B), _ptr(X), _ld(X),
                                                  ctypes.byref(o), ctypes.byref(rep), _stream(stream)))
    return rep


def lu_trailing_update(update, A, B, C, m, n, k, *, stream=None):
    """C := C - A B (FP32 column-major tensors: A (k, lda), B (n, ldb), C (n, ldc))."""
    return _check("lu_trailing_update", lib().lu_trailing_update(update, m, n, k, _ptr(A), _ld(A), _ptr(B),
                                                                  _ld(B), _ptr(C), _ld(C), _stream(stream)))


def lu_trailing_update_f64(update, A, B, C, m, n, k, *, stream=None):
    """C := C - A B (FP64 column-major tensors); update LU_UPDATE_NATIVE or LU_UPDATE_F64EMU (k <= 64)."""
    return _check("lu_trailing_update_f64", lib().lu_trailing_update_f64(update, m, n, k, _ptr(A), _ld(A), _ptr(B),
                                                                          _ld(B), _ptr(C), _ld(C), _stream(stream)))


def lu_workspace_size(routine: str, n: int, nrhs: int, dtype_code: int) -> int:
    return lib().lu_workspace_size(routine.encode(), n, nrhs, dtype_code)


def lu_status_string(code: int) -> str:
    return lib().lu_status_string(code).decode()


def lu_last_device_status(stream=None, reset=False) -> int:
    return lib().lu_last_device_status(_stream(stream), int(bool(reset)))


def lu_get_status(stream=None) -> int:
    """LU_OK or LU_ERR_TIMEOUT recorded by a bounded device wait (synchronizes the stream)."""
    return lib().lu_get_status(_stream(stream))


def lu_update_timing(enable: bool) -> int:
    return lib().lu_update_timing(int(bool(enable)))


def lu_update_timing_read():
    """(launches, total_ms, flops, bytes) of the timed trailing-update launches."""
    n = ctypes.c_longlong()
    ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check("lu_update_timing_read", lib().lu_update_timing_read(ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                                                 ctypes.byref(by)))
    return n.value, ms.value, fl.value, by.value


class TraceEvent(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("step", ctypes.c_int), ("stream", ctypes.c_int),
                ("t_start_ms", ctypes.c_float), ("t_end_ms", ctypes.c_float)]


def lu_trace(enable: bool) -> int:
    return lib().lu_trace(int(bool(enable)))


def lu_trace_read(max_events: int = 1 << 20):
    """Recorded launches as dicts (kind name, step, stream, start/end ms), then cleared."""
    buf = (TraceEvent * max_events)()
    n = lib().lu_trace_read(buf, max_events)
    _check("lu_trace_read", n if n < 0 else 0)
    return [dict(kind=LU_TRACE_KINDS[e.kind], step=e.step, stream=e.stream, t0=e.t_start_ms, t1=e.t_end_ms)
            for e in buf[:n]]


class CtaEvent(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("step", ctypes.c_int), ("cta", ctypes.c_int), ("smid", ctypes.c_int),
                ("tiles", ctypes.c_int), ("pad", ctypes.c_int), ("t0_ns", ctypes.c_ulonglong), ("t1_ns", ctypes.c_ulonglong)]


def lu_cta_trace(capacity: int) -> int:
    """Install (capacity > 0) or remove (0) the per-CTA trace ring of the factorization kernels."""
    return _check("lu_cta_trace", lib().lu_cta_trace(int(capacity)))


def lu_cta_trace_read(max_events: int = 1 << 20):
    """(records made, list of dicts: kind name, step, cta, smid, tiles, t0/t1 in globaltimer ns); clears the ring."""
    buf = (CtaEvent * max_events)()
    made = lib().lu_cta_trace_read(buf, max_events)
    _check("lu_cta_trace_read", made if made < 0 else 0)
    return made, [dict(kind=LU_TRACE_KINDS[e.kind], step=e.step, cta=e.cta, smid=e.smid, tiles=e.tiles, t0=e.t0_ns,
                       t1=e.t1_ns) for e in buf[:min(made, max_events)]]


def lu_wait_selftest(bound_ns: int, stream=None) -> int:
    """Status recorded by a forward substitution whose first block is withheld (LU_ERR_TIMEOUT expected)."""
    return lib().lu_wait_selftest(int(bound_ns), _stream(stream))


def lu_div_selftest(dtype_code: int, count: int, seed: int = 1, stream=None) -> int:
    """Pairs on which the substitutions' quotient differs from IEEE division (0 expected)."""
    return lib().lu_div_selftest(dtype_code, int(count), int(seed), _stream(stream))


def lu_peak_probe(kind: int, iters: int, stream=None):
    """(TFLOP/s, ms) of one throughput-probe launch (PROBE_DFMA, PROBE_FFMA or PROBE_DMMA)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check("lu_peak_probe", lib().lu_peak_probe(kind, int(iters), ctypes.byref(tf), ctypes.byref(ms), _stream(stream)))
    return tf.value, ms.value


def lu_kernel_launches() -> int:
    return lib().lu_kernel_launches()


def lu_version() -> str:
    return lib().lu_version().decode()


def to_colmajor(M, ld=None):
    """Row-major (m, n) torch matrix -> column-major (n, ld) tensor (copy)."""
    import torch
    m, n = M.shape
    ld = m if ld is None else ld
    T = torch.zeros((n, ld), dtype=M.dtype, device=M.device)
    T[:, :m] = M.t()
    return T


def from_colmajor(T, m=None):
    """Inverse of to_colmajor: column-major (n, ld) tensor -> row-major (m, n) matrix."""
    m = T.shape[1] if m is None else m
    return T[:, :m].t().contiguous()


def _opts_dict(o):
    return {"nb": o.nb, "nb_inner": o.nb_inner, "panel_ctas": o.panel_ctas, "lookahead": o.lookahead, "update": o.update,
            "update_ctas": o.update_ctas, "sm_share": o.sm_share, "tile": o.tile, "early_term": o.early_term}


def lu_autotune(dtype_code, n, *, update=LU_UPDATE_NATIVE, budget_ms=0.0, stream=None):
    """Time candidate plans for lu_factor of order n and record the fastest in the
    tuning table (synchronizes the stream).  Returns {"opts": ..., "ms", "candidates"}."""
    r = TuneResult()
    _check("lu_autotune", lib().lu_autotune(dtype_code, n, update, float(budget_ms), ctypes.byref(r), _stream(stream)))
    return {"opts": _opts_dict(r.opts), "ms": r.ms, "candidates": r.candidates}


def lu_autotune_batched(dtype_code, ns, max_n, *, stream=None):
    """Time the batched panel widths on scratch matrices of the orders in ns (device int32)."""
    r = TuneResult()
    _check("lu_autotune_batched", lib().lu_autotune_batched(dtype_code, ns.shape[0], _ptr(ns), max_n, ctypes.byref(r),
                                                            _stream(stream)))
    return {"opts": _opts_dict(r.opts), "ms": r.ms, "candidates": r.candidates}


def lu_plan_info(dtype_code, n, *, nb=0, nb_inner=0, panel_ctas=0, lookahead=0, update=LU_UPDATE_NATIVE, update_ctas=0,
                 sm_share=0, tile=0, early_term=0):
    """(status, plan dict) of the plan lu_factor would run for these options (no CUDA call);
    status 0 = every panel fits, LU_ERR_UNSUPPORTED = one does not."""
    o = LuOpts(nb, nb_inner, panel_ctas, lookahead, update, 0, update_ctas, sm_share, tile, early_term)
    p = LuOpts()
    rc = lib().lu_plan_info(dtype_code, n, ctypes.byref(o), ctypes.byref(p))
    if rc < 0 and rc > -100:
        raise LuError("lu_plan_info", rc)
    return rc, _opts_dict(p)


def lu_tune_get(kind, dtype_code, n, *, update=LU_UPDATE_NATIVE):
    """The table's options for (kind, dtype, update, n) as a dict, or None."""
    o = LuOpts()
    return _opts_dict(o) if lib().lu_tune_get(kind, dtype_code, update, n, ctypes.byref(o)) else None


def lu_tune_put(kind, dtype_code, n, *, nb=0, nb_inner=0, panel_ctas=0, lookahead=0, update=LU_UPDATE_NATIVE,
                update_ctas=0, tile=0, ms=0.0):
    o = LuOpts(nb, nb_inner, panel_ctas, lookahead, update, 0, update_ctas, 0, tile)
    return _check("lu_tune_put", lib().lu_tune_put(kind, dtype_code, update, n, ctypes.byref(o), float(ms)))


def lu_tune_save(path) -> int:
    rc = lib().lu_tune_save(os.fsencode(path))
    if rc < 0:
        raise LuError("lu_tune_save", rc)
    return rc


def lu_tune_load(path) -> int:
    rc = lib().lu_tune_load(os.fsencode(path))
    if rc < 0:
        raise LuError("lu_tune_load", rc)
    return rc


def lu_tune_count() -> int:
    return lib().lu_tune_count()


def lu_tune_clear() -> None:
    lib().lu_tune_clear()
