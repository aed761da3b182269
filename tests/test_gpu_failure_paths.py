"""Failure paths of the C ABI on the GPU, made without faulting the device:
a bounded device-side wait that runs out (NL_ETIMEOUT, context intact), a
device allocation that fails (NL_ENOMEM, from the library's allocation test
hook), and the iterate returned when Newton does not converge (the one with
the smallest ||F||)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16051_gb300 import nl
from tests.conftest import newton_counts_agree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()


def _solve_raw(s, mode):
    x = np.empty(s.N)
    st = nl.lib().nl_solve(s._h, None, 1e-10, nl.MODES[mode], x.ctypes.data)
    return st, x


@pytest.mark.parametrize("cluster", [0, -1])
@pytest.mark.parametrize("mode", ["IR16", "GMRESIR16"])
def test_triangular_solve_wait_runs_out(cluster, mode):
    """wait_limit < 0 makes every wait of the half-precision triangular
    solves give up at once, whatever the producer does: the cluster solve
    (cluster = 0, N = 4096) and the global-memory solve (-1) record the
    timeout in their error word, every CTA returns, and the solve reports
    NL_ETIMEOUT.  The context stays usable: a solve on another handle, and
    on the same handle after its wait limit is restored, converge as the
    oracle does."""
    N, c = 4096, 0.9
    with nl.Solver(N, c, trsv_cluster=cluster, wait_limit=-1) as s:
        st, _ = _solve_raw(s, mode)
        assert st == nl.NL_ETIMEOUT, nl.STATUS_NAMES[st]
        assert "gave up" in nl.last_error()
        assert s.stats()["status"] == nl.NL_ETIMEOUT
    torch.cuda.synchronize()  # the device answers
    _, ro = O.newton(512, c, mode, tol=1e-10)
    with nl.Solver(512, c, trsv_cluster=cluster) as s:
        x, st = s.solve(tol=1e-10, mode=mode)
        assert st == nl.NL_OK and newton_counts_agree(s.stats()["newton_iters"], ro)


def test_allocation_failure_returns_enomem():
    """The allocation test hook fails the next device allocation: nl_create
    returns NL_ENOMEM and no handle; the first FP64-LU solve of a live handle
    (which allocates the double Jacobian) returns NL_ENOMEM and leaves the
    handle usable; with the hook spent both succeed."""
    L = nl.lib()
    h = nl._P()
    assert L.nl_debug_fail_allocs(1) == nl.NL_OK
    assert L.nl_create(256, 0.9, None, nl.ctypes.byref(h)) == nl.NL_ENOMEM
    assert not h.value
    assert "cudaMalloc" in nl.last_error()
    with nl.Solver(256, 0.9) as s:
        assert L.nl_debug_fail_allocs(1) == nl.NL_OK
        st, _ = _solve_raw(s, "FP64LU")
        assert st == nl.NL_ENOMEM
        x, st = s.solve(mode="FP64LU")
        assert st == nl.NL_OK
        x2, st = s.solve(mode="GMRESIR16")
        assert st == nl.NL_OK and np.max(np.abs(x - x2)) <= 1e-10 * np.max(np.abs(x))
    assert L.nl_debug_fail_allocs(0) == nl.NL_OK


@pytest.mark.parametrize("c,scale,maxit", [(0.999, 6.0, 7), (0.99, 4.5, 6), (0.9999, 1.0, 3)])
def test_best_iterate_on_not_converged(c, scale, maxit):
    """On NL_ENOTCONV the returned x is the iterate with the smallest ||F||
    of the history (far-from-solution starts make the history non-monotone):
    its residual, computed by the oracle's F in double, is the smallest
    entry of the history times ||F(x0)||, and nl_stats_t.fnorm is that
    norm."""
    N = 128
    x0 = scale * np.ones(N)
    with nl.Solver(N, c, newton_maxit=maxit) as s:
        x, st = s.solve(tol=1e-10, mode="GMRESIR16", x0=x0)
        S = s.stats()
    assert st == nl.NL_ENOTCONV and S["newton_iters"] == maxit
    h = np.array(S["hist"])
    best = int(np.argmin(h))
    fx = np.linalg.norm(O.F(N, c, x))
    assert abs(fx - h[best] * S["fnorm0"]) <= 1e-12 * S["fnorm0"] + 1e-9 * fx, (h, fx)
    assert abs(S["fnorm"] - h[best] * S["fnorm0"]) <= 1e-15 * S["fnorm0"]
    if best == 0:
        assert np.array_equal(x, x0)
    # the oracle returns its own best iterate by the same rule
    xo, ro = O.newton(N, c, "GMRESIR16", tol=1e-10, x0=x0, newton_maxit=maxit)
    fo = np.linalg.norm(O.F(N, c, xo))
    assert abs(fo - min(ro["hist"]) * np.linalg.norm(O.F(N, c, x0))) <= 1e-9 * fo + 1e-14


@pytest.mark.parametrize("gemm", [3, 5])
def test_persistent_grouped_lu_wait_runs_out(gemm):
    """The persistent grouped LU's dependency waits are bounded: with the poll
    limit set to give up at the first unmet poll, the off-diagonal tasks that
    start while their diagonal block is being factored give up, the launch
    completes, nl_lu_grouped returns NL_ETIMEOUT, and with the default limit
    the next call on the same context factors the same matrices correctly
    (bitwise the three-launch grouped LU with the same update)."""
    Ns = [1500, 300, 90]
    mats = [O.fl16(O.jacobian(N, 0.9, 1.0 + 0.3 * np.sin(np.arange(N)) ** 2).astype(np.float32).astype(np.float64))
            for N in Ns]

    def run(g):
        As, lds, ips = [], [], []
        for M in mats:
            N = M.shape[0]
            ld = ((N + 63) // 64) * 64
            a = np.zeros((N, ld), dtype=np.float16)
            a[:, :N] = M.astype(np.float16)
            As.append(torch.as_tensor(a, device="cuda"))
            lds.append(ld)
            ips.append(torch.empty(N, dtype=torch.int32, device="cuda"))
        flags = nl.lu_grouped(Ns, As, lds, ips, nb=64, gemm=g)
        torch.cuda.synchronize()
        return [A.cpu().numpy()[:, :n] for A, n in zip(As, Ns)], flags

    nl.grouped_wait_limit(-1)
    try:
        with pytest.raises(nl.NLError) as e:
            run(gemm)
        assert e.value.status == nl.NL_ETIMEOUT
    finally:
        nl.grouped_wait_limit(0)
    out, flags = run(gemm)
    ref, rflags = run(1 if gemm == 3 else 2)
    assert not flags.any() and not rflags.any()
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)
