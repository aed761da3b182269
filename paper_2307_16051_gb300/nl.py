"""ctypes binding of libnewton3p.so (the C ABI in include/newton3p.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Device arrays may be passed as torch tensors (their
``data_ptr()`` is used) or as integer addresses.  If the library cannot be
loaded the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

NL_OK, NL_EINVAL, NL_ENOMEM, NL_ENOTCONV, NL_ESINGULAR, NL_ENUMERIC, NL_ETIMEOUT, NL_ECUDA = range(8)
STATUS_NAMES = ["NL_OK", "NL_EINVAL", "NL_ENOMEM", "NL_ENOTCONV", "NL_ESINGULAR", "NL_ENUMERIC", "NL_ETIMEOUT",
                "NL_ECUDA"]
NL_FP64LU, NL_IR16, NL_GMRESIR16, NL_IR16_GMRES, NL_F32, NL_F16 = 0, 1, 2, 3, 4, 5
MODES = {"FP64LU": NL_FP64LU, "IR16": NL_IR16, "GMRESIR16": NL_GMRESIR16, "IR16_GMRES": NL_IR16_GMRES,
         "F32": NL_F32, "F16": NL_F16}
MAX_HIST = 128


class NLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("eta_j", ctypes.c_double), ("ir_maxit", ctypes.c_int), ("gmres_restart", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("gmres_maxcycles", ctypes.c_int), ("newton_maxit", ctypes.c_int),
                ("tau_a", ctypes.c_double), ("lu_nb", ctypes.c_int), ("trailing_gemm", ctypes.c_int),
                ("lu_path", ctypes.c_int), ("trsv_cluster", ctypes.c_int), ("lu_stream", ctypes.c_int),
                ("ir_variant", ctypes.c_int), ("gmres_factors32", ctypes.c_int), ("lu16_arith", ctypes.c_int),
                ("wait_limit", ctypes.c_int), ("scale_fp16", ctypes.c_int), ("fft_f", ctypes.c_int),
                ("lu_lookahead", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("mode", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("lu_nb", ctypes.c_int), ("fnorm0", ctypes.c_double), ("fnorm", ctypes.c_double),
                ("hist", ctypes.c_double * MAX_HIST), ("lin_iters", ctypes.c_int * MAX_HIST),
                ("lin_outer", ctypes.c_int * MAX_HIST), ("lin_failed", ctypes.c_int * MAX_HIST),
                ("lin_relres", ctypes.c_double * MAX_HIST), ("t_total_ms", ctypes.c_double),
                ("t_f_ms", ctypes.c_double), ("t_jac_ms", ctypes.c_double), ("t_lu_ms", ctypes.c_double),
                ("t_lin_ms", ctypes.c_double), ("gpu_launches", ctypes.c_int), ("lu_pivoted", ctypes.c_int),
                ("lu_tune_count", ctypes.c_int), ("lu_tune_nb", ctypes.c_int * 4), ("lu_tune_ms", ctypes.c_float * 4),
                ("reserved", ctypes.c_int * 5)]


BATCH_MAX_TUNE = 48  # NL_BATCH_MAX_TUNE


class BatchInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("converged", ctypes.c_int), ("parked_lu", ctypes.c_int),
                ("parked_ir", ctypes.c_int), ("newton_rounds", ctypes.c_int), ("ir_rounds", ctypes.c_int),
                ("lu_nb", ctypes.c_int), ("trailing_gemm", ctypes.c_int), ("gpu_launches", ctypes.c_int),
                ("graph_nodes_step", ctypes.c_int), ("graph_nodes_ir", ctypes.c_int), ("tune_count", ctypes.c_int),
                ("tune_bucket", ctypes.c_int * BATCH_MAX_TUNE), ("tune_nb", ctypes.c_int * BATCH_MAX_TUNE),
                ("tune_gemm", ctypes.c_int * BATCH_MAX_TUNE), ("tune_ms", ctypes.c_double * BATCH_MAX_TUNE),
                ("nbuckets", ctypes.c_int), ("bucket_nmax", ctypes.c_int * 8), ("bucket_count", ctypes.c_int * 8),
                ("bucket_nb", ctypes.c_int * 8), ("bucket_gemm", ctypes.c_int * 8), ("bucket_cached", ctypes.c_int * 8),
                ("lu16_ms", ctypes.c_double),
                ("t_total_ms", ctypes.c_double), ("t_graph_ms", ctypes.c_double), ("t_single_ms", ctypes.c_double),
                ("reserved", ctypes.c_int * 16)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int), ("mode", ctypes.c_int),
                ("tol", ctypes.c_double), ("starve_ms", ctypes.c_int), ("priority_n", ctypes.c_int),
                ("policy", ctypes.c_int), ("solver", Config),
                ("reserved", ctypes.c_int * 8)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("N", ctypes.c_int), ("c", ctypes.c_double), ("t_arrive_s", ctypes.c_double),
                ("t_admit_s", ctypes.c_double), ("t_done_s", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("newton_iters", ctypes.c_int), ("handle_reused", ctypes.c_int), ("reserved", ctypes.c_int * 6)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("bytes_held", ctypes.c_int64), ("bytes_peak", ctypes.c_int64), ("inflight_peak", ctypes.c_int),
                ("handles_created", ctypes.c_int), ("handles_evicted", ctypes.c_int), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("span_s", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("reserved", ctypes.c_int * 8)]


_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p
_i64, _dbl, _int = ctypes.c_int64, ctypes.c_double, ctypes.c_int

# name -> (restype, argtypes); kept in the order of include/newton3p.h
SIGNATURES = {
    "nl_config_default": (_int, [ctypes.POINTER(Config)]),
    "nl_create": (_int, [_i64, _dbl, ctypes.POINTER(Config), ctypes.POINTER(_P)]),
    "nl_set_stream": (_int, [_P, _P]),
    "nl_solve": (_int, [_P, _P, _dbl, _int, _P]),
    "nl_solve_device": (_int, [_P, _P, _dbl, _int, _P]),
    "nl_stats": (_int, [_P, ctypes.POINTER(Stats)]),
    "nl_device_bytes": (_i64, [_P]),
    "nl_destroy": (None, [_P]),
    "nl_last_error": (ctypes.c_char_p, []),
    "nl_version": (ctypes.c_char_p, []),
    "nl_kernel_timing": (_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "nl_debug_fail_allocs": (_int, [_int]),
    "nl_k_residual": (_int, [_i64, _dbl, _P, _P, _int, _dbl, _P, _P, _P, _P, _P]),
    "nl_k_jacobian": (_int, [_i64, _dbl, _P, _P, _i64, _P, _i64, _P]),
    "nl_k_residual_fft": (_int, [_i64, _dbl, _P, _P, _int, _dbl, _P, _P, _P, _P, _P]),
    "nl_k_jacobian_scaled": (_int, [_i64, _dbl, _P, _P, _i64, _P, _i64, _P, _P]),
    "nl_k_jacobian64": (_int, [_i64, _dbl, _P, _P, _i64, _P]),
    "nl_lu16": (_int, [_i64, _P, _i64, _P, _int, _int, _int, ctypes.POINTER(ctypes.c_int32), _P]),
    "nl_lu64": (_int, [_i64, _P, _i64, _P, _int, _int, ctypes.POINTER(ctypes.c_int32), _P]),
    "nl_lusolve16": (_int, [_i64, _P, _i64, _P, _P, _P]),
    "nl_lusolve64": (_int, [_i64, _P, _i64, _P, _P, _P]),
    "nl_lu32": (_int, [_i64, _P, _i64, _P, _int, ctypes.POINTER(ctypes.c_int32), _P]),
    "nl_lusolve32": (_int, [_i64, _P, _i64, _P, _P, _P]),
    "nl_lusolve16h": (_int, [_i64, _P, _i64, _P, _P, _P]),
    "nl_k_gemv_residual": (_int, [_i64, _P, _i64, _P, _P, _P, _P, _P]),
    "nl_k_gemv_residual_noalloc": (_int, [_i64, _P, _i64, _P, _P, _P, _P, _P]),
    "nl_k_div_round16": (_int, [_i64, _P, _P, _P, _P]),
    "nl_k_gemm16_update": (_int, [_i64, _i64, _i64, _P, _i64, _P, _i64, _P, _i64, _int, _P]),
    "nl_linsolve16": (_int, [_i64, _P, _i64, _P, _i64, _P, _P, _P, _dbl, _int, _int, _int, _dbl, _int,
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), _P]),
    "nl_batch_create": (_int, [_int, _P, _P, ctypes.POINTER(Config), ctypes.POINTER(_P)]),
    "nl_batch_solve": (_int, [_P, _P, _dbl, _int, _P]),
    "nl_batch_solve_device": (_int, [_P, _P, _dbl, _int, _P]),
    "nl_batch_stats": (_int, [_P, _int, ctypes.POINTER(Stats)]),
    "nl_batch_info": (_int, [_P, ctypes.POINTER(BatchInfo)]),
    "nl_batch_set_stream": (_int, [_P, _P]),
    "nl_batch_device_bytes": (_i64, [_P]),
    "nl_batch_destroy": (None, [_P]),
    "nl_set_c": (_int, [_P, _dbl]),
    "nl_footprint_bytes": (_i64, [_i64, _int, ctypes.POINTER(Config)]),
    "nl_server_config_default": (_int, [ctypes.POINTER(ServerConfig)]),
    "nl_server_create": (_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]),
    "nl_server_submit": (_int, [_P, _i64, _dbl, _dbl, ctypes.POINTER(ctypes.c_int64)]),
    "nl_server_start": (_int, [_P]),
    "nl_server_result": (_int, [_P, _i64, _int, _P, ctypes.POINTER(Stats), ctypes.POINTER(RequestInfo)]),
    "nl_server_drain": (_int, [_P, _dbl]),
    "nl_server_info": (_int, [_P, ctypes.POINTER(ServerInfo)]),
    "nl_server_destroy": (None, [_P]),
    "nl_lu_grouped": (_int, [_int, _P, _P, _P, _P, _int, _int, _int, _P, _P]),
    "nl_debug_grouped_task_times": (_int, [_int, _P]),
    "nl_debug_grouped_wait_limit": (_int, [ctypes.c_longlong]),
    "nl_k_update32": (_int, [_i64, _i64, _i64, _P, _i64, _P, _i64, _P, _i64, _P]),
    "nl_lusolve_grouped": (_int, [_int, _P, _P, _P, _P, _P, _int, _P]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libnewton3p.so (building it in-tree if missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise NLError(NL_ECUDA, f"CUDA library not found at {path}")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype, f.argtypes = res, args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().nl_last_error().decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def check(status, allow=()):
    if status != NL_OK and status not in allow:
        raise NLError(status, last_error())
    return status


def config(**kw) -> Config:
    c = Config()
    check(lib().nl_config_default(ctypes.byref(c)))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def kernel_timing(kernel_class=None):
    """(launches, total_ms) of the class timed so far; then time `kernel_class`."""
    cnt = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    check(lib().nl_kernel_timing(kernel_class.encode() if kernel_class else None, ctypes.byref(cnt), ctypes.byref(ms)))
    return cnt.value, ms.value


class Solver:
    """Owns one nl_solver handle (device state for one (N, c) problem)."""

    def __init__(self, N: int, c: float, stream=None, **cfg):
        self._h = _P()
        check(lib().nl_create(int(N), float(c), ctypes.byref(config(**cfg)), ctypes.byref(self._h)))
        self.N, self.c = int(N), float(c)
        if stream is not None:
            check(lib().nl_set_stream(self._h, _stream(stream)))

    def close(self):
        if self._h:
            lib().nl_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, tol=1e-10, mode="GMRESIR16", x0=None, out=None):
        """Host-memory solve (nl_solve).  Returns (x, status).  x0 and out may
        be numpy arrays in pinned memory (float64, N)."""
        x = np.empty(self.N) if out is None else out
        if x.dtype != np.float64 or x.size != self.N or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a contiguous float64 array of length N")
        x0p = None
        if x0 is not None:
            x0 = np.ascontiguousarray(x0, dtype=np.float64)
            x0p = x0.ctypes.data
        st = lib().nl_solve(self._h, x0p, float(tol), MODES[mode] if isinstance(mode, str) else int(mode),
                            x.ctypes.data)
        check(st, allow=(NL_ENOTCONV,))
        return x, st

    def solve_device(self, x_out, tol=1e-10, mode="GMRESIR16", x0=None):
        st = lib().nl_solve_device(self._h, _ptr(x0), float(tol), MODES[mode] if isinstance(mode, str) else int(mode),
                                   _ptr(x_out))
        return check(st, allow=(NL_ENOTCONV,))

    def stats(self) -> dict:
        s = Stats()
        check(lib().nl_stats(self._h, ctypes.byref(s)))
        n = s.newton_iters
        return dict(status=s.status, mode=s.mode, newton_iters=n, lu_nb=s.lu_nb, fnorm0=s.fnorm0, fnorm=s.fnorm,
                    hist=list(s.hist[: n + 1]), lin_iters=list(s.lin_iters[:n]), lin_outer=list(s.lin_outer[:n]),
                    lin_failed=list(s.lin_failed[:n]), lin_relres=list(s.lin_relres[:n]),
                    t_total_ms=s.t_total_ms, t_f_ms=s.t_f_ms, t_jac_ms=s.t_jac_ms, t_lu_ms=s.t_lu_ms,
                    t_lin_ms=s.t_lin_ms, gpu_launches=s.gpu_launches, lu_pivoted=s.lu_pivoted,
                    lu_tune=[(s.lu_tune_nb[k], s.lu_tune_ms[k]) for k in range(s.lu_tune_count)])

    def device_bytes(self) -> int:
        return lib().nl_device_bytes(self._h)


def _stats_dict(s: Stats) -> dict:
    n = s.newton_iters
    return dict(status=s.status, mode=s.mode, newton_iters=n, lu_nb=s.lu_nb, fnorm0=s.fnorm0, fnorm=s.fnorm,
                hist=list(s.hist[: n + 1]), lin_iters=list(s.lin_iters[:n]), lin_outer=list(s.lin_outer[:n]),
                lin_failed=list(s.lin_failed[:n]), lin_relres=list(s.lin_relres[:n]),
                t_total_ms=s.t_total_ms, gpu_launches=s.gpu_launches, lu_pivoted=s.lu_pivoted)


class Batch:
    """Owns one nl_batch handle: many (N, c) instances solved together."""

    def __init__(self, Ns, cs, stream=None, **cfg):
        self.N = np.ascontiguousarray(Ns, dtype=np.int64)
        self.c = np.ascontiguousarray(cs, dtype=np.float64)
        if self.N.shape != self.c.shape or self.N.ndim != 1:
            raise ValueError("Ns and cs must be 1-D arrays of the same length")
        self.count = int(self.N.size)
        self.off = np.concatenate([[0], np.cumsum(self.N)]).astype(np.int64)
        self._h = _P()
        check(lib().nl_batch_create(self.count, self.N.ctypes.data, self.c.ctypes.data, ctypes.byref(config(**cfg)),
                                    ctypes.byref(self._h)))
        if stream is not None:
            check(lib().nl_batch_set_stream(self._h, _stream(stream)))

    def close(self):
        if self._h:
            lib().nl_batch_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, tol=1e-10, mode="IR16_GMRES", x0=None):
        """Host-memory solve (nl_batch_solve).  Returns (list of x, status)."""
        x = np.empty(int(self.off[-1]))
        x0p = None
        if x0 is not None:
            x0 = np.ascontiguousarray(x0, dtype=np.float64)
            x0p = x0.ctypes.data
        st = lib().nl_batch_solve(self._h, x0p, float(tol), MODES[mode] if isinstance(mode, str) else int(mode),
                                  x.ctypes.data)
        check(st, allow=(NL_ENOTCONV, NL_ENUMERIC, NL_ESINGULAR))
        return [x[self.off[i]:self.off[i + 1]] for i in range(self.count)], st

    def solve_device(self, x_out, tol=1e-10, mode="IR16_GMRES", x0=None):
        st = lib().nl_batch_solve_device(self._h, _ptr(x0), float(tol),
                                         MODES[mode] if isinstance(mode, str) else int(mode), _ptr(x_out))
        return check(st, allow=(NL_ENOTCONV, NL_ENUMERIC, NL_ESINGULAR))

    def stats(self, i: int) -> dict:
        s = Stats()
        check(lib().nl_batch_stats(self._h, int(i), ctypes.byref(s)))
        return _stats_dict(s)

    def info(self) -> dict:
        b = BatchInfo()
        check(lib().nl_batch_info(self._h, ctypes.byref(b)))
        d = {k: getattr(b, k) for k, _ in BatchInfo._fields_ if not k.startswith(("tune_", "bucket_", "reserved"))}
        d["tune_count"] = b.tune_count
        # (nb, gemm, ms, bucket) of every timed candidate
        d["tune"] = [(b.tune_nb[k], b.tune_gemm[k], b.tune_ms[k], b.tune_bucket[k]) for k in range(b.tune_count)]
        d["buckets"] = [{"nmax": b.bucket_nmax[k], "count": b.bucket_count[k], "nb": b.bucket_nb[k],
                         "gemm": b.bucket_gemm[k], "cached": b.bucket_cached[k]} for k in range(b.nbuckets)]
        return d

    def device_bytes(self) -> int:
        return lib().nl_batch_device_bytes(self._h)


# ---------------------------------------------------------------- kernels --

def k_residual(N, c, x, F, r, fnorm, u=None, u_is_double=False, scale=0.0, x_out=None, stream=None):
    return check(lib().nl_k_residual(N, c, _ptr(x), _ptr(u), int(u_is_double), float(scale), _ptr(x_out), _ptr(F),
                                     _ptr(r), _ptr(fnorm), _stream(stream)))


def k_jacobian(N, c, r, J32, ld32, J16, ld16, stream=None):
    return check(lib().nl_k_jacobian(N, c, _ptr(r), _ptr(J32), ld32, _ptr(J16), ld16, _stream(stream)))


def k_residual_fft(N, c, x, F, r, fnorm, u=None, u_is_double=False, scale=0.0, x_out=None, stream=None):
    return check(lib().nl_k_residual_fft(N, c, _ptr(x), _ptr(u), int(u_is_double), float(scale), _ptr(x_out),
                                         _ptr(F), _ptr(r), _ptr(fnorm), _stream(stream)))


def k_jacobian_scaled(N, c, r, J32, ld32, J16, ld16, rs, stream=None):
    check(lib().nl_k_jacobian_scaled(N, c, _ptr(r), _ptr(J32), ld32, _ptr(J16), ld16, _ptr(rs), _stream(stream)))


def k_jacobian64(N, c, r, J64, ld, stream=None):
    return check(lib().nl_k_jacobian64(N, c, _ptr(r), _ptr(J64), ld, _stream(stream)))


def lu16(N, A16, ld, ipiv, nb=0, gemm=0, path=0, stream=None):
    info = ctypes.c_int32(0)
    st = lib().nl_lu16(N, _ptr(A16), ld, _ptr(ipiv), nb, gemm, path, ctypes.byref(info), _stream(stream))
    check(st, allow=(NL_ESINGULAR,))
    return info.value


def lu64(N, A, ld, ipiv, nb=0, path=0, stream=None):
    info = ctypes.c_int32(0)
    st = lib().nl_lu64(N, _ptr(A), ld, _ptr(ipiv), nb, path, ctypes.byref(info), _stream(stream))
    check(st, allow=(NL_ESINGULAR,))
    return info.value


def lusolve16(N, LU16, ld, ipiv, b, stream=None):
    return check(lib().nl_lusolve16(N, _ptr(LU16), ld, _ptr(ipiv), _ptr(b), _stream(stream)))


def lusolve64(N, LU, ld, ipiv, b, stream=None):
    return check(lib().nl_lusolve64(N, _ptr(LU), ld, _ptr(ipiv), _ptr(b), _stream(stream)))


def lu32(N, A, ld, ipiv, nb=0, stream=None):
    info = ctypes.c_int32(0)
    st = lib().nl_lu32(N, _ptr(A), ld, _ptr(ipiv), nb, ctypes.byref(info), _stream(stream))
    check(st, allow=(NL_ESINGULAR,))
    return info.value


def lusolve32(N, LU, ld, ipiv, b, stream=None):
    return check(lib().nl_lusolve32(N, _ptr(LU), ld, _ptr(ipiv), _ptr(b), _stream(stream)))


def lusolve16h(N, LU16, ld, ipiv, b16, stream=None):
    return check(lib().nl_lusolve16h(N, _ptr(LU16), ld, _ptr(ipiv), _ptr(b16), _stream(stream)))


def k_gemv_residual(N, A, ld, b, u, r, rnorm, stream=None):
    return check(lib().nl_k_gemv_residual(N, _ptr(A), ld, _ptr(b), _ptr(u), _ptr(r), _ptr(rnorm), _stream(stream)))


def k_gemv_residual_noalloc(N, A, ld, b, u, r, rnorm, stream=None):
    """nl_k_gemv_residual without any device allocation (fixed in-library scratch)."""
    return check(lib().nl_k_gemv_residual_noalloc(N, _ptr(A), ld, _ptr(b), _ptr(u), _ptr(r), _ptr(rnorm),
                                                  _stream(stream)))


def k_gemm16_update(M, Nc, K, A, lda, B, ldb, C, ldc, gemm=1, stream=None):
    return check(lib().nl_k_gemm16_update(M, Nc, K, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, gemm, _stream(stream)))


def k_update32(M, Nc, K, A, lda, B, ldb, C, ldc, stream=None):
    return check(lib().nl_k_update32(M, Nc, K, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, _stream(stream)))


def linsolve16(N, J32, ld32, LU16, ld16, ipiv, b, u, eta=1e-4, maxit=20, solver=0, m=30, gtol=1e-4, gcycles=10,
               stream=None):
    stats = (ctypes.c_int32 * 4)()
    rel = ctypes.c_double(0.0)
    check(lib().nl_linsolve16(N, _ptr(J32), ld32, _ptr(LU16), ld16, _ptr(ipiv), _ptr(b), _ptr(u), eta, maxit, solver,
                              m, gtol, gcycles, stats, ctypes.byref(rel), _stream(stream)))
    return dict(iters=stats[0], outer=stats[1], failed=stats[2], converged=stats[3], relres=rel.value)


def grouped_wait_limit(polls: int):
    """Test hook: polls before a persistent grouped-LU wait gives up (0 default, < 0 at once)."""
    check(lib().nl_debug_grouped_wait_limit(int(polls)))


def grouped_task_times(enable=True) -> dict:
    """Per-task timing of the persistent grouped LU since the previous call
    (nl_debug_grouped_task_times); then switch it on or off."""
    out = (ctypes.c_double * 9)()
    check(lib().nl_debug_grouped_task_times(int(enable), ctypes.cast(out, _P)))
    res = {}
    for k, name in enumerate(("diag", "quad", "tile")):
        n = out[3 * k]
        res[name] = {"tasks": int(n), "wait_us": out[3 * k + 1] / n if n else 0.0,
                     "work_us": out[3 * k + 2] / n if n else 0.0}
    return res


def lu_grouped(Ns, As, lds, ipivs, fp64=False, nb=0, gemm=0, stream=None):
    """Grouped LU (nl_lu_grouped) of device matrices; returns the per-matrix flags."""
    n = len(Ns)
    Na = np.ascontiguousarray(Ns, dtype=np.int64)
    lda = np.ascontiguousarray(lds, dtype=np.int64)
    Ap = np.ascontiguousarray([_ptr(a) for a in As], dtype=np.uint64)
    Pp = np.ascontiguousarray([_ptr(p) for p in ipivs], dtype=np.uint64)
    flags = np.zeros(n, dtype=np.int32)
    check(lib().nl_lu_grouped(n, Na.ctypes.data, Ap.ctypes.data, lda.ctypes.data, Pp.ctypes.data, int(fp64), nb, gemm,
                              flags.ctypes.data, _stream(stream)))
    return flags


def lusolve_grouped(Ns, LUs, lds, ipivs, bs, fp64=False, stream=None):
    """Grouped triangular solves (nl_lusolve_grouped), in place on the device vectors bs."""
    n = len(Ns)
    Na = np.ascontiguousarray(Ns, dtype=np.int64)
    lda = np.ascontiguousarray(lds, dtype=np.int64)
    Lp = np.ascontiguousarray([_ptr(a) for a in LUs], dtype=np.uint64)
    Pp = np.ascontiguousarray([_ptr(p) for p in ipivs], dtype=np.uint64)
    Bp = np.ascontiguousarray([_ptr(b) for b in bs], dtype=np.uint64)
    return check(lib().nl_lusolve_grouped(n, Na.ctypes.data, Lp.ctypes.data, lda.ctypes.data, Pp.ctypes.data,
                                          Bp.ctypes.data, int(fp64), _stream(stream)))


def footprint_bytes(N, mode="IR16_GMRES", **cfg) -> int:
    return lib().nl_footprint_bytes(int(N), MODES[mode] if isinstance(mode, str) else int(mode),
                                    ctypes.byref(config(**cfg)))


class Server:
    """Owns one nl_server: requests admitted by device-memory footprint and
    solved concurrently on their own streams."""

    def __init__(self, budget_bytes=64 << 30, max_inflight=8, mode="IR16_GMRES", tol=1e-10, starve_ms=250,
                 priority_n=1024, policy=1, **cfg):
        sc = ServerConfig()
        check(lib().nl_server_config_default(ctypes.byref(sc)))
        sc.hbm_budget_bytes = int(budget_bytes)
        sc.max_inflight = int(max_inflight)
        sc.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        sc.tol = float(tol)
        sc.starve_ms = int(starve_ms)
        sc.priority_n = int(priority_n)
        sc.policy = int(policy)
        for k, v in cfg.items():
            setattr(sc.solver, k, v)
        self._h = _P()
        check(lib().nl_server_create(ctypes.byref(sc), ctypes.byref(self._h)))
        self.sizes = {}

    def submit(self, N, c, arrival_s=-1.0) -> int:
        rid = ctypes.c_int64(0)
        check(lib().nl_server_submit(self._h, int(N), float(c), float(arrival_s), ctypes.byref(rid)))
        self.sizes[rid.value] = int(N)
        return rid.value

    def start(self):
        check(lib().nl_server_start(self._h))

    def result(self, rid, wait=True):
        """(x, stats dict, request info dict) of request rid."""
        N = self.sizes[rid]
        x = np.empty(N)
        s = Stats()
        ri = RequestInfo()
        check(lib().nl_server_result(self._h, int(rid), int(wait), x.ctypes.data, ctypes.byref(s), ctypes.byref(ri)))
        info = {k: getattr(ri, k) for k, _ in RequestInfo._fields_ if k != "reserved"}
        return x, _stats_dict(s), info

    def drain(self, timeout_s=0.0):
        return check(lib().nl_server_drain(self._h, float(timeout_s)), allow=(NL_ETIMEOUT,))

    def info(self) -> dict:
        si = ServerInfo()
        check(lib().nl_server_info(self._h, ctypes.byref(si)))
        return {k: getattr(si, k) for k, _ in ServerInfo._fields_ if k != "reserved"}

    def close(self):
        if self._h:
            lib().nl_server_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def k_div_round16(n, a, b, out, stream=None):
    """out = fl16(fl32(a / b)) as the LU's multiplier rounding computes it."""
    return check(lib().nl_k_div_round16(int(n), _ptr(a), _ptr(b), _ptr(out), _stream(stream)))
