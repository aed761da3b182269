"""The optional scaling of the Jacobian into the binary16 range before the
down-cast (nl_config.scale_fp16; Section 2.3 on underflow when rounding to
half precision): J_h = I_s^h(R J32) with power-of-two row factors R, the
solves applied to R times their right-hand side.  Checked against the
oracle run with the same scaling."""
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


def rel_inf(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _jacobians(N, c, x, scaled):
    """GPU J32, J16 bits and row factors at x (r from the GPU residual)."""
    dev = "cuda"
    xd = torch.as_tensor(x, device=dev)
    F = torch.empty(N, device=dev, dtype=torch.float64)
    r = torch.empty(N, device=dev, dtype=torch.float64)
    fn = torch.empty(1, device=dev, dtype=torch.float64)
    nl.k_residual(N, c, xd, F, r, fn)
    ld = (N + 63) // 64 * 64
    J32 = torch.empty(N, ld, device=dev, dtype=torch.float32)
    J16 = torch.empty(N, ld, device=dev, dtype=torch.float16)
    if scaled:
        rs = torch.empty(N, device=dev, dtype=torch.float32)
        nl.k_jacobian_scaled(N, c, r, J32, ld, J16, ld, rs)
    else:
        rs = None
        nl.k_jacobian(N, c, r, J32, ld, J16, ld)
    torch.cuda.synchronize()
    return (J32[:, :N].cpu().numpy(), J16[:, :N].cpu().view(torch.int16).numpy().view(np.uint16),
            None if rs is None else rs.cpu().numpy())


@pytest.mark.parametrize("N,c", [(1, 0.5), (100, 0.0), (513, 0.9), (4096, 0.99), (8192, 0.999999)])
def test_scaled_jacobian_bits(N, c):
    """rs is the oracle's power-of-two row factor, J32 is unscaled, and every
    J16 entry is fl16(rs_i J32_ij) bit for bit (the product is exact)."""
    x = np.linspace(1.0, 2.0, N) if N > 1 else np.ones(1)
    J32, J16, rs = _jacobians(N, c, x, True)
    J32u, J16u, _ = _jacobians(N, c, x, False)
    assert np.array_equal(J32, J32u)
    assert np.array_equal(rs, O.row_scales(N, c, x).astype(np.float32))
    want = O.f16_bits_from_f32((J32 * rs[:, None]).astype(np.float32)).reshape(N, N)
    assert np.array_equal(J16, want)
    assert np.all(np.abs(J16.view(np.float16).astype(np.float64)) <= 2.0 ** 13)


def test_scaling_lifts_entries_out_of_the_subnormal_range():
    """At N = 8192 about half of the entries of I_s^h(J32) lie below the
    binary16 minimum normal 2^-14 (about 6.1e-5; at N = 32768 nearly all
    off-diagonal ones do); scaled by 2^12, only the smallest corner entries
    (mu_i / (mu_i + mu_j) near 1/(2N)) still do."""
    N, c = 8192, 0.99
    x = np.ones(N)
    _, J16u, _ = _jacobians(N, c, x, False)
    _, J16s, _ = _jacobians(N, c, x, True)
    def sub_frac(bits):
        e = (bits >> 10) & 0x1F
        m = bits & 0x3FF
        return float(np.mean((e == 0) & (m != 0)))
    fu, fs = sub_frac(J16u), sub_frac(J16s)
    print(f"subnormal fraction of J16 at N={N}, c={c}: unscaled {fu:.3f}, scaled {fs:.3f}")
    assert fu > 0.4 and fs < 0.01 and fs < fu / 50


@pytest.mark.parametrize("mode", ["IR16", "GMRESIR16", "IR16_GMRES"])
@pytest.mark.parametrize("N,c", [(63, 0.5), (512, 0.9), (1000, 0.99), (2048, 0.9999)])
def test_scaled_newton_matches_oracle(mode, N, c):
    """Newton with the scaled factorisation: Newton counts as the oracle's
    with the same scaling, linear counts within one (one outer correction at
    c = .9999), and the solution within the Newton tolerance of the oracle's
    FP64-LU solution (kappa-amplified for c = .9999, as for the unscaled
    modes)."""
    with nl.Solver(N, c, scale_fp16=1) as s:
        x, status = s.solve(tol=1e-10, mode=mode)
        st = s.stats()
    om = "IR16GM" if mode == "IR16_GMRES" else mode
    _, ro = O.newton(N, c, om, tol=1e-10, scale_fp16=1)
    x64, r64 = O.newton(N, c, "FP64LU", tol=1e-10)
    assert status == nl.NL_OK and ro["status"] == 0
    assert newton_counts_agree(st["newton_iters"], ro), (st["hist"], ro["hist"])
    if c >= 0.9999:
        for a, b in zip(st["lin_outer"], ro["lin_outer"]):
            assert abs(a - b) <= 1, (st["lin_outer"], ro["lin_outer"])
    else:
        for a, b in zip(st["lin_iters"], ro["lin_iters"]):
            assert abs(a - b) <= 1, (st["lin_iters"], ro["lin_iters"])
    kappa = 1.0 / math.sqrt(1.0 - c)
    tol = 1e-10 if c <= 0.99 else 1e-10 + 10.0 * kappa * max(st["hist"][-1], r64["hist"][-1])
    err = rel_inf(x, x64)
    print(f"scaled {mode} N={N} c={c}: newton {st['newton_iters']} lin {st['lin_iters']} err vs FP64 oracle {err:.2e}")
    assert err <= tol


def test_scaling_off_is_the_default_path():
    """scale_fp16 = 0 is the unscaled path bit for bit."""
    with nl.Solver(777, 0.99) as a, nl.Solver(777, 0.99, scale_fp16=0) as b:
        xa, _ = a.solve(mode="GMRESIR16")
        xb, _ = b.solve(mode="GMRESIR16")
    assert np.array_equal(xa, xb)


def test_scaling_rejected_for_f16_column():
    with nl.Solver(64, 0.5, scale_fp16=1) as s:
        st = nl.lib().nl_solve(s._h, None, 1e-10, nl.NL_F16, np.empty(64).ctypes.data)
        assert st == nl.NL_EINVAL


def test_scaled_large_n32768():
    """N = 32768, c = .99, GMRES-IR16 with the scaled factorisation: checked
    by what holds at any size (the oracle's F at the GPU iterate meets the
    tolerance; the exact discrete moment identity)."""
    N, c = 32768, 0.99
    with nl.Solver(N, c, scale_fp16=1) as s:
        x, status = s.solve(tol=1e-10, mode="GMRESIR16")
        st = s.stats()
    assert status == nl.NL_OK and st["lu_pivoted"] == 0
    f = np.linalg.norm(O.F(N, c, x))
    assert f <= 1e-10 * st["fnorm0"] * 1.0001
    m = c / (2 * N) * np.sum(x)
    assert abs(m - (1 - math.sqrt(1 - c))) <= 1e-9 / math.sqrt(1 - c)
    print(f"scaled N=32768: newton {st['newton_iters']} lin {st['lin_iters']}")
