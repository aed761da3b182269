"""ctypes binding for the CPU oracle in ``oracle.c``.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` load this module; the product path never
does.  It compiles ``oracle.c`` with gcc on first use (or via ``build()``)
and exposes numpy-friendly wrappers.  Nothing here imports the CUDA package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FP64LU, IR16, GMRESIR16, F32, F16, IR16GM = 0, 1, 2, 3, 4, 5
MODES = {"FP64LU": FP64LU, "IR16": IR16, "GMRESIR16": GMRESIR16, "F32": F32, "F16": F16, "IR16GM": IR16GM}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (plain IEEE arithmetic:
    no -ffast-math, no multiply-add contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("ir_maxit", ctypes.c_int), ("gmres_m", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("gmres_cycles", ctypes.c_int),
                ("newton_maxit", ctypes.c_int), ("tau_a", ctypes.c_double), ("ir_variant", ctypes.c_int),
                ("lu_nb", ctypes.c_int), ("scale_fp16", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("hist", ctypes.c_double * 128), ("lin_iters", ctypes.c_int * 128),
                ("lin_outer", ctypes.c_int * 128), ("lin_failed", ctypes.c_int * 128),
                ("lin_relres", ctypes.c_double * 128), ("lu_info", ctypes.c_int * 128)]


class LinStat(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("failed", ctypes.c_int),
                ("converged", ctypes.c_int), ("relres", ctypes.c_double)]


_D = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_F = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_I = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_H = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
_i64, _dbl, _int = ctypes.c_int64, ctypes.c_double, ctypes.c_int


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "orc_fl16": (_dbl, [_dbl]),
                "orc_f16_bits": (ctypes.c_uint16, [_dbl]),
                "orc_f16_value": (_dbl, [ctypes.c_uint16]),
                "orc_fl16_array": (None, [_i64, _D, _D]),
                "orc_f16_bits_array_f32": (None, [_i64, _F, _H]),
                "orc_F": (None, [_i64, _dbl, _D, _D]),
                "orc_jacobian": (None, [_i64, _dbl, _D, _D]),
                "orc_norm2": (_dbl, [_i64, _D]),
                "orc_lu64": (_int, [_i64, _D, _I]),
                "orc_lu32": (_int, [_i64, _F, _I]),
                "orc_lu16": (_int, [_i64, _D, _I, ctypes.POINTER(_int)]),
                "orc_lu16_dev": (_int, [_i64, _i64, _D, _I, ctypes.POINTER(_int)]),
                "orc_lu16_recip": (_int, [_i64, _D, _I, ctypes.POINTER(_int)]),
                "orc_lusolve64": (None, [_i64, _D, _I, _D]),
                "orc_lusolve32": (None, [_i64, _F, _I, _F]),
                "orc_lusolve_fly": (None, [_i64, _D, _I, _F]),
                "orc_lusolve16": (None, [_i64, _D, _I, _D]),
                "orc_gmres": (_int, [_i64, _F, _D, _I, _D, _D, _int, _dbl, _int]),
                "orc_linsolve": (None, [_i64, _F, _D, _I, _F, _F, _dbl, _int, _int, _int, _dbl, _int,
                                        ctypes.POINTER(LinStat)]),
                "orc_linsolve_scaled": (None, [_i64, _F, _D, _I, ctypes.c_void_p, _F, _F, _dbl, _int, _int, _int,
                                               _dbl, _int, ctypes.POINTER(LinStat)]),
                "orc_row_scales": (None, [_i64, _dbl, _D, _D]),
                "orc_newton": (_int, [_i64, _dbl, _int, ctypes.c_void_p, _dbl, ctypes.POINTER(Params), _D,
                                      ctypes.POINTER(Result)]),
                "orc_num_threads": (_int, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype, f.argtypes = res, args
            _lib = L
    return _lib


# --------------------------------------------------------------------------
# numpy wrappers
# --------------------------------------------------------------------------

def fl16(x) -> np.ndarray:
    """Round doubles to the nearest binary16 value (RNE), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(a)
    lib().orc_fl16_array(a.size, a.ravel(), out.ravel())
    return out


def f16_bits_from_f32(x) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.float32).ravel()
    out = np.empty(a.size, dtype=np.uint16)
    lib().orc_f16_bits_array_f32(a.size, a, out)
    return out


def F(N: int, c: float, x) -> np.ndarray:
    """Residual of eq. (3.2) [hmid] in double."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(N)
    lib().orc_F(N, c, x, out)
    return out


def jacobian(N: int, c: float, x) -> np.ndarray:
    """Analytic Jacobian of eq. (3.2) in double, N x N row-major."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty((N, N))
    lib().orc_jacobian(N, c, x, out)
    return out


def norm2(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().orc_norm2(v.size, v)


def lu64(A):
    """Partial-pivot LU in double.  Returns (LU, ipiv, info)."""
    a = np.array(A, dtype=np.float64, order="C", copy=True)
    N = a.shape[0]
    ipiv = np.empty(N, dtype=np.int32)
    info = lib().orc_lu64(N, a, ipiv)
    return a, ipiv, info


def lu32(A):
    a = np.array(A, dtype=np.float32, order="C", copy=True)
    N = a.shape[0]
    ipiv = np.empty(N, dtype=np.int32)
    info = lib().orc_lu32(N, a, ipiv)
    return a, ipiv, info


def lu16(A16):
    """Partial-pivot LU in binary16 arithmetic.  A16 must hold binary16
    values (float64 or float16 array).  Returns (LU as float64, ipiv, info,
    overflow)."""
    a = np.array(A16, dtype=np.float64, order="C", copy=True)
    N = a.shape[0]
    ipiv = np.empty(N, dtype=np.int32)
    ovf = _int(0)
    info = lib().orc_lu16(N, a, ipiv, ctypes.byref(ovf))
    return a, ipiv, info, bool(ovf.value)


def lu16_recip(A16):
    """As lu16 with each multiplier fl16(a_ik * fl16(1 / a_kk)) (the column
    scaled by the rounded reciprocal of the pivot).  Returns (LU, ipiv, info,
    overflow)."""
    a = np.array(A16, dtype=np.float64, order="C", copy=True)
    N = a.shape[0]
    ipiv = np.empty(N, dtype=np.int32)
    ovf = _int(0)
    info = lib().orc_lu16_recip(N, a, ipiv, ctypes.byref(ovf))
    return a, ipiv, info, bool(ovf.value)


def lu16_dev(A16, nb):
    """Binary16-storage / binary32-arithmetic LU with rounding period nb.
    Returns (LU as float64 holding binary16 values, ipiv, info, overflow)."""
    a = np.array(A16, dtype=np.float64, order="C", copy=True)
    N = a.shape[0]
    ipiv = np.empty(N, dtype=np.int32)
    ovf = _int(0)
    info = lib().orc_lu16_dev(N, int(nb), a, ipiv, ctypes.byref(ovf))
    return a, ipiv, info, bool(ovf.value)


def lusolve64(LU, ipiv, b):
    x = np.array(b, dtype=np.float64, copy=True)
    lib().orc_lusolve64(LU.shape[0], np.ascontiguousarray(LU), np.ascontiguousarray(ipiv, np.int32), x)
    return x


def lusolve32(LU, ipiv, b):
    x = np.array(b, dtype=np.float32, copy=True)
    lib().orc_lusolve32(LU.shape[0], np.ascontiguousarray(LU, np.float32), np.ascontiguousarray(ipiv, np.int32), x)
    return x


def lusolve_fly(LU16, ipiv, b):
    """Eq. (2.16): fp16 factors promoted on the fly, single-precision solve."""
    x = np.array(b, dtype=np.float32, copy=True)
    lib().orc_lusolve_fly(LU16.shape[0], np.ascontiguousarray(LU16, np.float64),
                          np.ascontiguousarray(ipiv, np.int32), x)
    return x


def lusolve16(LU16, ipiv, b16):
    x = np.array(b16, dtype=np.float64, copy=True)
    lib().orc_lusolve16(LU16.shape[0], np.ascontiguousarray(LU16, np.float64),
                        np.ascontiguousarray(ipiv, np.int32), x)
    return x


def gmres(A32, LU16, ipiv, r, m=30, tol=1e-4, cycles=10):
    """Left-preconditioned GMRES(m) with d0 = 0.  Returns (d, arnoldi_steps)."""
    N = A32.shape[0]
    d = np.empty(N)
    steps = lib().orc_gmres(N, np.ascontiguousarray(A32, np.float32), np.ascontiguousarray(LU16, np.float64),
                            np.ascontiguousarray(ipiv, np.int32), np.ascontiguousarray(r, np.float64), d,
                            m, tol, cycles)
    return d, steps


SOLVER_IR_FLY, SOLVER_IR_CHEAP, SOLVER_GMRES = 0, 1, 2


def linsolve(A32, LU16, ipiv, b, solver=SOLVER_IR_FLY, eta=1e-4, maxit=20, m=30, gtol=1e-4, gcycles=10, rs=None):
    """IR / GMRES-IR from u0 = 0.  rs: row factors R when LU16 factors R A
    (scaled into the binary16 range), else None.  Returns (u, LinStat as dict)."""
    N = A32.shape[0]
    u = np.empty(N, dtype=np.float32)
    st = LinStat()
    rsp = None
    if rs is not None:
        rs = np.ascontiguousarray(rs, np.float64)
        rsp = rs.ctypes.data_as(ctypes.c_void_p)
    lib().orc_linsolve_scaled(N, np.ascontiguousarray(A32, np.float32), np.ascontiguousarray(LU16, np.float64),
                              np.ascontiguousarray(ipiv, np.int32), rsp, np.ascontiguousarray(b, np.float32), u,
                              eta, maxit, solver, m, gtol, gcycles, ctypes.byref(st))
    return u, {k: getattr(st, k) for k, _ in LinStat._fields_}


def row_scales(N: int, c: float, x) -> np.ndarray:
    """Power-of-two row factors that scale J into the binary16 range."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(N)
    lib().orc_row_scales(N, c, x, out)
    return out


DEFAULT_LU_NB = 128


def default_params(paper: bool = False) -> dict:
    """Parameter set.  paper=True: eta_J = 1e-6 and at most 10 Newton steps
    (Section 3.1 and Tables 2-3); otherwise eta_J = 1e-4 and 30 steps.
    lu_nb selects the half-precision factorisation's arithmetic: 0 = every
    operation in binary16, > 0 = binary16 storage with binary32 arithmetic
    and rounding period lu_nb (the GPU's model)."""
    return dict(eta=1e-6 if paper else 1e-4, ir_maxit=20, gmres_m=30, gmres_tol=1e-4, gmres_cycles=10,
                newton_maxit=10 if paper else 30, tau_a=0.0, ir_variant=0, lu_nb=DEFAULT_LU_NB, scale_fp16=0)


def newton(N: int, c: float, mode="IR16", tol=1e-10, x0=None, **overrides):
    """Run the oracle Newton iteration.  Returns (x, result dict)."""
    p = default_params(overrides.pop("paper", False))
    p.update(overrides)
    prm = Params(**p)
    res = Result()
    x = np.empty(N)
    if x0 is not None:
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        ptr = x0.ctypes.data_as(ctypes.c_void_p)
    else:
        ptr = None
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    lib().orc_newton(N, c, m, ptr, tol, ctypes.byref(prm), x, ctypes.byref(res))
    n = res.newton_iters
    out = dict(status=res.status, newton_iters=n, hist=list(res.hist[: n + 1]),
               lin_iters=list(res.lin_iters[:n]), lin_outer=list(res.lin_outer[:n]),
               lin_failed=list(res.lin_failed[:n]), lin_relres=list(res.lin_relres[:n]),
               lu_info=list(res.lu_info[:n]))
    return x, out


def num_threads() -> int:
    return lib().orc_num_threads()
