"""The residual of eq. (3.2) evaluated in O(N log N) through an FFT
convolution (Section 3), nl_k_residual_fft and nl_config.fft_f, against the
oracle's direct double sum (orc_F) and the GPU's direct kernel."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16051_gb300 import nl
from tests.conftest import newton_counts_agree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep_n4096.json")
GOLDEN_X = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep_n4096_x.npy")
SWEEP = (0.5, 0.9, 0.99, 0.9999, 0.999999)


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()


def _residual(fn, N, c, x, u=None, scale=0.0):
    dev = "cuda"
    xd = torch.as_tensor(x, device=dev)
    F = torch.empty(N, device=dev, dtype=torch.float64)
    r = torch.empty(N, device=dev, dtype=torch.float64)
    nrm = torch.empty(1, device=dev, dtype=torch.float64)
    xo = torch.empty(N, device=dev, dtype=torch.float64) if u is not None else None
    ud = torch.as_tensor(u, device=dev) if u is not None else None
    fn(N, c, xd, F, r, nrm, u=ud, u_is_double=False, scale=scale, x_out=xo)
    torch.cuda.synchronize()
    return (F.cpu().numpy(), r.cpu().numpy(), nrm.item(), None if xo is None else xo.cpu().numpy())


@pytest.mark.parametrize("N", [1, 2, 3, 7, 100, 1000, 1023, 1025, 4096, 32768])
@pytest.mark.parametrize("c", [0.5, 0.999999])
def test_fft_residual_matches_oracle(N, c):
    """At x0 = ones and at a non-trivial positive x: every F_i within
    1e-13 max|r| of the oracle's direct sum (the rounding of a length-L
    double FFT, L = 2^ceil(log2 2N)), r likewise, ||F|| within 1e-12
    relative; the GPU's direct kernel agrees to the same bound."""
    for x in (np.ones(N), 1.0 + 0.5 * np.sin(np.arange(N) * 0.37) ** 2):
        Fo = O.F(N, c, x)
        ro = x - Fo
        F, r, nrm, _ = _residual(nl.k_residual_fft, N, c, x)
        Fd, rd, nd, _ = _residual(nl.k_residual, N, c, x)
        scale = np.max(np.abs(ro))
        assert np.max(np.abs(F - Fo)) <= 1e-13 * scale, (N, c, np.max(np.abs(F - Fo)))
        assert np.max(np.abs(r - ro)) <= 1e-13 * scale
        assert np.max(np.abs(F - Fd)) <= 1e-13 * scale
        assert abs(nrm - np.linalg.norm(Fo)) <= 1e-12 * np.linalg.norm(Fo) + 1e-13 * scale
        print(f"N={N} c={c}: max|F_fft - F_oracle| = {np.max(np.abs(F - Fo)):.2e} (max|r| {scale:.2f}), "
              f"direct {np.max(np.abs(Fd - Fo)):.2e}")


def test_fft_residual_fused_update_and_determinism():
    """x_out = x + scale u with the direct kernel's rounding (bitwise), and two
    calls give the same bits."""
    N, c = 3000, 0.99
    g = np.random.default_rng(3)
    x = 1.0 + g.random(N)
    u = g.standard_normal(N).astype(np.float32)
    F1, r1, n1, xo1 = _residual(nl.k_residual_fft, N, c, x, u, 0.37)
    F2, r2, n2, xo2 = _residual(nl.k_residual_fft, N, c, x, u, 0.37)
    _, _, _, xod = _residual(nl.k_residual, N, c, x, u, 0.37)
    assert np.array_equal(xo1, xod) and np.array_equal(F1, F2) and n1 == n2
    Fo = O.F(N, c, xod)
    assert np.max(np.abs(F1 - Fo)) <= 1e-13 * np.max(np.abs(xod - Fo))


@pytest.mark.parametrize("N", [1, 63, 129, 1000, 2049])
@pytest.mark.parametrize("mode", ["FP64LU", "IR16", "GMRESIR16"])
def test_newton_with_fft_residual(N, mode):
    """Newton with F through the FFT (fft_f = 1; the direct sum, fft_f = -1,
    below N = 4096 by default): the oracle's Newton counts and solution."""
    c = 0.99
    with nl.Solver(N, c, fft_f=1) as s:
        x, status = s.solve(tol=1e-10, mode=mode)
        st = s.stats()
    xo, ro = O.newton(N, c, mode, tol=1e-10)
    assert status == nl.NL_OK and newton_counts_agree(st["newton_iters"], ro), (st["hist"], ro["hist"])
    assert np.max(np.abs(x - xo)) <= 1e-10 * np.max(np.abs(xo))


@pytest.mark.skipif(not (os.path.exists(GOLDEN) and os.path.exists(GOLDEN_X)), reason="golden sweep files missing")
@pytest.mark.parametrize("c", list(SWEEP))
def test_sweep_n4096_with_fft_residual(c):
    """The N = 4096 sweep (GMRES-IR16) with F through the FFT: the oracle's
    counts and, element by element, its FP64-LU solution (1e-10 for c <= .99,
    kappa-scaled beyond, as for the direct residual)."""
    gold = json.load(open(GOLDEN))
    ro = gold["cases"][f"{c}/GMRESIR16"]
    x64 = np.load(GOLDEN_X)[SWEEP.index(c)]
    with nl.Solver(4096, c, fft_f=1) as s:
        x, status = s.solve(tol=1e-10, mode="GMRESIR16")
        st = s.stats()
    assert status == nl.NL_OK and newton_counts_agree(st["newton_iters"], ro)
    kappa = 1.0 / math.sqrt(1.0 - c)
    tol = 1e-10 if c <= 0.99 else 1e-10 + 10.0 * kappa * max(st["hist"][-1], ro["hist"][-1])
    err = np.max(np.abs(x - x64)) / np.max(np.abs(x64))
    print(f"fft F, N=4096 c={c}: newton {st['newton_iters']} err {err:.2e}")
    assert err <= tol


def test_fft_default_switch():
    """fft_f = 0 (default) takes the FFT from N = 4096: the same bits as fft_f = 1
    there, the direct sum's bits (fft_f = -1) below."""
    for N, same_as in ((4096, 1), (2048, -1)):
        with nl.Solver(N, 0.99) as a, nl.Solver(N, 0.99, fft_f=same_as) as b:
            xa, _ = a.solve(mode="GMRESIR16")
            xb, _ = b.solve(mode="GMRESIR16")
        assert np.array_equal(xa, xb), N
