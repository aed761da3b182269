"""The allocation-free residual entry point (nl_k_gemv_residual_noalloc).

Callers that cannot allocate device memory (code inside a fixed pool that
owns all of the device memory, a plug-in that must not grow the device
footprint) use this
variant; it must give the same residual and norm as nl_k_gemv_residual.
Collected last so that a failure here cannot hide any other test's result.
"""
import numpy as np
import pytest

from paper_2307_16051_gb300 import nl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _case(N, seed):
    g = np.random.default_rng(seed)
    ld = ((N + 63) // 64) * 64
    A = torch.zeros((N, ld), device="cuda", dtype=torch.float32)
    if N <= 4096:
        A[:, :N] = torch.as_tensor(g.standard_normal((N, N)).astype(np.float32), device="cuda")
    else:  # the largest case (4 GiB) drawn on the device from a seeded generator
        gd = torch.Generator(device="cuda")
        gd.manual_seed(seed)
        A[:, :N] = torch.randn((N, N), device="cuda", dtype=torch.float32, generator=gd)
    u = torch.zeros(ld, device="cuda", dtype=torch.float32)
    u[:N] = torch.as_tensor(g.standard_normal(N).astype(np.float32), device="cuda")
    b = torch.as_tensor(g.standard_normal(N).astype(np.float32), device="cuda")
    return A, ld, b, u


@pytest.mark.parametrize("N,seed,with_b", [(1000, 1, True), (4096, 2, True), (1001, 4, True), (1001, 5, False),
                                           (32768, 6, True)])
def test_noalloc_matches_allocating_entry_point_twice(N, seed, with_b):
    """Sizes with a ragged last block of eight rows (1001), no right side
    (b = NULL: r = -A u), and the largest N, whose partial sums fill the
    scratch up to the counter word."""
    assert torch.cuda.is_available(), "needs a CUDA device"
    A, ld, b, u = _case(N, seed)
    if not with_b:
        b = None
    r_ref = torch.empty(N, device="cuda", dtype=torch.float32)
    n_ref = torch.empty(1, device="cuda", dtype=torch.float64)
    nl.k_gemv_residual(N, A, ld, b, u, r_ref, n_ref)
    for _ in range(2):  # two calls in a row: the shared scratch must not leak state
        r = torch.full((N,), float("nan"), device="cuda", dtype=torch.float32)
        n = torch.full((1,), float("nan"), device="cuda", dtype=torch.float64)
        nl.k_gemv_residual_noalloc(N, A, ld, b, u, r, n)
        torch.cuda.synchronize()
        # deterministic kernels: the same bits as the allocating path
        assert torch.equal(r, r_ref)
        assert n.item() == n_ref.item()
    del A


def test_noalloc_without_norm_output():
    """rnorm_dev = NULL: only the residual vector is written."""
    N = 777
    A, ld, b, u = _case(N, 7)
    r_ref = torch.empty(N, device="cuda", dtype=torch.float32)
    n_ref = torch.empty(1, device="cuda", dtype=torch.float64)
    nl.k_gemv_residual(N, A, ld, b, u, r_ref, n_ref)
    r = torch.full((N,), float("nan"), device="cuda", dtype=torch.float32)
    nl.k_gemv_residual_noalloc(N, A, ld, b, u, r, None)
    torch.cuda.synchronize()
    assert torch.equal(r, r_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    A, ld, b, u = _case(8, 3)
    r = torch.empty(8, device="cuda", dtype=torch.float32)
    n = torch.empty(1, device="cuda", dtype=torch.float64)
    st = nl.lib().nl_k_gemv_residual_noalloc(32769, A.data_ptr(), 32832, b.data_ptr(), u.data_ptr(), r.data_ptr(),
                                             n.data_ptr(), None)
    assert st == nl.NL_EINVAL and "32768" in nl.last_error()
