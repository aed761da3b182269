"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point that include/newton3p.h declares; argument
validation and the no-device path return the documented statuses."""
import os
import re

import pytest

from paper_2307_16051_gb300 import nl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:[\w\s\*]+?)\b(nl_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("nl_create", "nl_solve", "nl_stats", "nl_destroy", "nl_lu16", "nl_lusolve16", "nl_linsolve16"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = nl.lib()
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
    assert set(declared_symbols()) <= set(nl.SIGNATURES), "binding lacks a signature"


def test_version_and_defaults():
    L = nl.lib()
    assert b"sm_103a" in L.nl_version()
    c = nl.config()
    assert c.eta_j == 1e-4 and c.ir_maxit == 20 and c.gmres_restart == 30 and c.gmres_tol == 1e-4
    assert c.newton_maxit == 30 and c.tau_a == 0.0


def test_invalid_arguments_rejected_before_device_use():
    L = nl.lib()
    h = nl._P()
    for N, c in [(0, 0.5), (-3, 0.5), (10, 1.0), (10, -0.1), (10, float("nan")), (40000, 0.5)]:
        assert L.nl_create(N, c, None, nl.ctypes.byref(h)) == nl.NL_EINVAL
    assert L.nl_create(10, 0.5, None, None) == nl.NL_EINVAL
    assert L.nl_solve(None, None, 1e-10, 1, None) == nl.NL_EINVAL
    assert L.nl_config_default(None) == nl.NL_EINVAL
    assert L.nl_stats(None, None) == nl.NL_EINVAL
    assert "bad" in nl.last_error() or "NULL" in nl.last_error()
    L.nl_destroy(None)  # no-op
    for bad in ({"trsv_cluster": 3}, {"trsv_cluster": -2}, {"trsv_cluster": 32}, {"lu_path": 2}, {"lu_stream": 1},
                {"lu_stream": -2}, {"ir_variant": 2}, {"ir_variant": -1}, {"gmres_factors32": 2},
                {"gmres_factors32": -1}, {"lu16_arith": 2}, {"scale_fp16": 2}, {"scale_fp16": -1},
                {"scale_fp16": 1, "ir_variant": 1}, {"scale_fp16": 1, "gmres_factors32": 1},
                {"scale_fp16": 1, "lu16_arith": 1}, {"fft_f": 2}, {"fft_f": -2}, {"lu_lookahead": 1},
                {"lu_lookahead": -2}):
        assert L.nl_create(64, 0.5, nl.ctypes.byref(nl.config(**bad)), nl.ctypes.byref(h)) == nl.NL_EINVAL, bad
    # the two-precision kernel entries check their arguments before any device call
    assert L.nl_lu32(0, None, 0, None, 0, None, None) == nl.NL_EINVAL
    assert L.nl_lu32(64, 1, 64, 1, 24, None, None) == nl.NL_EINVAL  # nb not a multiple of 16
    assert L.nl_lusolve32(40000, 1, 40000, 1, 1, None) == nl.NL_EINVAL
    assert L.nl_lusolve16h(64, 1, 32, 1, 1, None) == nl.NL_EINVAL  # ld < N
    assert L.nl_lusolve16h(64, None, 64, 1, 1, None) == nl.NL_EINVAL
    assert L.nl_solve(None, None, 1e-10, nl.NL_F16, None) == nl.NL_EINVAL


def test_no_device_is_an_error_not_a_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = nl._P()
    assert nl.lib().nl_create(64, 0.5, None, nl.ctypes.byref(h)) == nl.NL_ECUDA
    with pytest.raises(nl.NLError):
        nl.Solver(64, 0.5)


def test_batch_arguments_validated():
    L = nl.lib()
    h = nl._P()
    import numpy as np
    for Ns, cs in [([], []), ([0], [0.5]), ([8193], [0.5]), ([10, 20], [0.5, 1.0]), ([10], [-0.5])]:
        N = np.ascontiguousarray(Ns, dtype=np.int64)
        c = np.ascontiguousarray(cs, dtype=np.float64)
        assert L.nl_batch_create(len(Ns), N.ctypes.data if len(Ns) else None, c.ctypes.data if len(cs) else None,
                                 None, nl.ctypes.byref(h)) == nl.NL_EINVAL
    # the batched path solves with the on-the-fly correction only
    N = np.ascontiguousarray([64], dtype=np.int64)
    c = np.ascontiguousarray([0.5], dtype=np.float64)
    assert L.nl_batch_create(1, N.ctypes.data, c.ctypes.data, nl.ctypes.byref(nl.config(ir_variant=1)),
                             nl.ctypes.byref(h)) == nl.NL_EINVAL
    assert L.nl_batch_create(1, N.ctypes.data, c.ctypes.data, nl.ctypes.byref(nl.config(gmres_factors32=1)),
                             nl.ctypes.byref(h)) == nl.NL_EINVAL
    assert L.nl_batch_create(1, N.ctypes.data, c.ctypes.data, nl.ctypes.byref(nl.config(lu16_arith=1)),
                             nl.ctypes.byref(h)) == nl.NL_EINVAL
    assert L.nl_batch_solve(None, None, 1e-10, nl.NL_IR16_GMRES, None) == nl.NL_EINVAL
    assert L.nl_batch_stats(None, 0, None) == nl.NL_EINVAL
    assert L.nl_lu_grouped(0, None, None, None, None, 0, 0, 0, None, None) == nl.NL_EINVAL
    assert L.nl_lusolve_grouped(0, None, None, None, None, None, 0, None) == nl.NL_EINVAL
    L.nl_batch_destroy(None)


def test_batch_no_device_is_an_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(nl.NLError):
        nl.Batch([64, 100], [0.5, 0.9])


def test_server_no_device_is_an_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(nl.NLError):
        nl.Server()
    assert nl.lib().nl_server_submit(None, 64, 0.5, 0.0, None) == nl.NL_EINVAL
    assert nl.lib().nl_server_create(None, None) == nl.NL_EINVAL
    assert nl.footprint_bytes(1024) > 6 * 1024 * 1024
    assert nl.footprint_bytes(1024, "FP64LU") > nl.footprint_bytes(1024) + 8 * 1024 * 1024
    assert nl.lib().nl_footprint_bytes(0, 1, None) == -1
    assert nl.lib().nl_footprint_bytes(64, 6, None) == -1  # no such mode
    # F16 needs nothing beyond the handle; F32 adds the single-precision solve's workspace
    assert nl.footprint_bytes(1024, "F16") == nl.footprint_bytes(1024, "IR16")
    assert nl.footprint_bytes(1024, "F32") > nl.footprint_bytes(1024, "IR16")
    # the single-precision factor copy: 4 N ld bytes more, and only for the GMRES-IR modes
    assert nl.footprint_bytes(1024, "GMRESIR16", gmres_factors32=1) >= nl.footprint_bytes(1024, "GMRESIR16") + 4 * 1024 * 1024
    assert nl.footprint_bytes(1024, "IR16", gmres_factors32=1) == nl.footprint_bytes(1024, "IR16")
    # the autotuning setting (-1) sizes the handle for its largest candidate (the two-level
    # outer block 512, with its single-precision shadow of the matrix)
    for N in (1, 700, 4096):
        assert nl.footprint_bytes(N, lu_nb=-1) == nl.footprint_bytes(N, lu_nb=512) > nl.footprint_bytes(N, lu_nb=128)
        assert nl.footprint_bytes(N, lu_nb=128) >= nl.footprint_bytes(N, lu_nb=32)
        assert nl.footprint_bytes(N, lu_nb=512) >= nl.footprint_bytes(N, lu_nb=128) + 4 * N * N


def test_test_hooks_and_scaled_jacobian_validate_arguments():
    L = nl.lib()
    assert L.nl_debug_fail_allocs(-1) == nl.NL_EINVAL
    assert L.nl_debug_fail_allocs(0) == nl.NL_OK
    # the scaled Jacobian needs its row-factor output; bad sizes are rejected first
    assert L.nl_k_jacobian_scaled(64, 0.5, 8, 8, 64, 8, 64, None, None) == nl.NL_EINVAL
    assert L.nl_k_jacobian_scaled(0, 0.5, 8, 8, 64, 8, 64, 8, None) == nl.NL_EINVAL
    c = nl.config()
    assert c.wait_limit == 0 and c.scale_fp16 == 0 and c.fft_f == 0
