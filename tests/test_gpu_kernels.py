"""Kernel-level parity of the CUDA path (through the C ABI) against the CPU
oracle, on seeded inputs spanning several tiles and ragged tails."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16051_gb300 import nl
from paper_2307_16051_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def T(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), device=dev(), dtype=dtype)


def ulp32(x):
    x = np.abs(np.asarray(x, np.float32))
    return np.spacing(np.maximum(x, np.float32(2.0 ** -126)))


# ---------------------------------------------------------------- K1 / K2 --

@pytest.mark.parametrize("N", [1, 7, 100, 517, 2048])
@pytest.mark.parametrize("c", [0.5, 0.99])
def test_residual_matches_oracle(N, c):
    g = np.random.default_rng(N)
    x = 1.0 + g.uniform(0.0, 1.0, N)
    u = g.standard_normal(N).astype(np.float32)
    scale = 0.37
    F = torch.empty(N, device=dev(), dtype=torch.float64)
    r = torch.empty_like(F)
    xo = torch.empty_like(F)
    fn = torch.empty(1, device=dev(), dtype=torch.float64)
    # plain evaluation
    nl.k_residual(N, c, T(x), F, r, fn)
    Fo = O.F(N, c, x)
    assert np.allclose(F.cpu().numpy(), Fo, rtol=1e-12, atol=1e-13)
    assert abs(fn.item() - np.linalg.norm(Fo)) <= 1e-12 * max(1.0, np.linalg.norm(Fo))
    # fused update x + scale * u
    nl.k_residual(N, c, T(x), F, r, fn, u=T(u), scale=scale, x_out=xo)
    xn = x + scale * u.astype(np.float64)
    assert np.array_equal(xo.cpu().numpy(), xn)
    Fo = O.F(N, c, xn)
    assert np.allclose(F.cpu().numpy(), Fo, rtol=1e-12, atol=1e-13)
    # r_i = 1/(1 - t_i) is what the Jacobian needs: F = x - r
    assert np.allclose(r.cpu().numpy(), xn - Fo, rtol=1e-12)


@pytest.mark.parametrize("N", [1, 9, 130, 1000])
def test_jacobian_matches_oracle(N):
    c = 0.99
    g = np.random.default_rng(10 + N)
    x = 1.0 + g.uniform(0.0, 1.0, N)
    ld = ((N + 63) // 64) * 64
    F = torch.empty(N, device=dev(), dtype=torch.float64)
    r = torch.empty_like(F)
    fn = torch.empty(1, device=dev(), dtype=torch.float64)
    nl.k_residual(N, c, T(x), F, r, fn)
    J32 = torch.full((N, ld), 7.0, device=dev(), dtype=torch.float32)
    J16 = torch.full((N, ld), 7.0, device=dev(), dtype=torch.float16)
    nl.k_jacobian(N, c, r, J32, ld, J16, ld)
    J32h = J32.cpu().numpy()
    J16h = J16.cpu().numpy()
    Jo = O.jacobian(N, c, x)
    ref32 = Jo.astype(np.float32)
    # single-precision formation: within 2 units in the last place of the
    # correctly rounded value (eq. (2.1): error O(u_s))
    err = np.abs(J32h[:, :N].astype(np.float64) - ref32.astype(np.float64))
    assert np.all(err <= 2 * ulp32(ref32) + 1e-30)
    # J_h = I_s^h(J32) exactly (round to nearest even, Section 2)
    bits = O.f16_bits_from_f32(J32h[:, :N])
    assert np.array_equal(bits.reshape(N, N), J16h[:, :N].view(np.uint16))
    assert np.all(J32h[:, N:] == 0) and np.all(J16h[:, N:] == 0)
    J64 = torch.full((N, ld), 7.0, device=dev(), dtype=torch.float64)
    nl.k_jacobian64(N, c, r, J64, ld)
    # double formation from the reciprocal table: a few units in the last place
    assert np.allclose(J64.cpu().numpy()[:, :N], Jo, rtol=2e-14, atol=1e-18)


# -------------------------------------------------------------- K3: LU16 --

def _lu16_gpu(A16, nb, gemm, path=0):
    N = A16.shape[0]
    ld = ((N + 63) // 64) * 64
    Ad = torch.zeros((N, ld), device=dev(), dtype=torch.float16)
    Ad[:, :N] = T(A16.astype(np.float16))
    ipiv = torch.empty(N, device=dev(), dtype=torch.int32)
    info = nl.lu16(N, Ad, ld, ipiv, nb=nb, gemm=gemm, path=path)
    return Ad.cpu().numpy()[:, :N].astype(np.float64), ipiv.cpu().numpy(), info


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("N,nb", [(1, 16), (16, 16), (37, 16), (100, 32), (200, 64), (333, 128), (517, 128)])
def test_lu16_simt_bit_exact_vs_oracle(N, nb, path):
    """SIMT trailing update: the GPU factorisation is operation-for-operation
    the oracle's binary16-storage / binary32-arithmetic elimination.  These
    matrices need row interchanges, so path 0 tries the no-interchange fast
    path, detects that, and refactors with interchanges."""
    A, _ = W.pivot_forcing_matrix(N, 1000 + N)
    A16 = O.fl16(A)
    LU, ipiv, info = _lu16_gpu(A16, nb, 1, path)
    LUo, ipivo, infoo, _ = O.lu16_dev(A16, nb)
    assert info == infoo == 0
    assert np.array_equal(ipiv, ipivo)
    assert np.array_equal(LU, LUo)


@pytest.mark.parametrize("N,nb", [(600, 128), (1000, 64), (77, 16), (300, 48), (129, 128), (255, 96)])
def test_lu16_simt_bit_exact_on_jacobian(N, nb):
    """The paper's Jacobian needs no interchanges: the fast path (path 0)
    and the interchanging path (path 1) both reproduce the oracle bit for bit."""
    c = 0.99
    x = np.ones(N)
    J16 = O.fl16(O.jacobian(N, c, x).astype(np.float32).astype(np.float64))
    LUo, ipivo, _, _ = O.lu16_dev(J16, nb)
    assert np.array_equal(ipivo, np.arange(N))
    for path in (0, 1):
        LU, ipiv, _ = _lu16_gpu(J16, nb, 1, path)
        assert np.array_equal(ipiv, ipivo) and np.array_equal(LU, LUo), path


@pytest.mark.parametrize("N,nb,gemm", [(1000, 128, 2), (4097, 128, 2), (700, 64, 1), (383, 96, 1)])
def test_lu16_streaming_panel_equals_two_launches(N, nb, gemm):
    """The streaming panel (one cooperative launch per panel, the off-diagonal
    solves one column behind the diagonal block) and the two-launch panel do
    the same fused multiply-adds in the same order: bitwise the same factors,
    on the paper's Jacobian and on a matrix whose fast path fails late."""
    c = 0.999
    J16 = O.fl16(O.jacobian(N, c, np.ones(N)).astype(np.float32).astype(np.float64))
    B, perm = W.pivot_forcing_matrix(min(N, 600), 17, margin=4.0)
    B = B[np.argsort(perm)]
    B[[B.shape[0] - 40, B.shape[0] - 30]] = B[[B.shape[0] - 30, B.shape[0] - 40]]
    for M in (J16, O.fl16(B)):
        res = [_lu16_gpu(M, nb, gemm, path) for path in (0, 2)]
        assert np.array_equal(res[0][1], res[1][1])
        assert np.array_equal(res[0][0], res[1][0])
        assert res[0][2] == res[1][2]


def test_lu16_fast_path_detects_late_interchange():
    """A matrix that needs exactly one interchange deep inside: the fast
    path must detect it and the result must equal the oracle's."""
    N = 300
    A, perm = W.pivot_forcing_matrix(N, 9, margin=4.0)
    B = A[np.argsort(perm)]                            # undo the permutation: diagonal pivots
    B[[250, 260]] = B[[260, 250]]                      # one late interchange
    A16 = O.fl16(B)
    LUo, ipivo, _, _ = O.lu16_dev(A16, 128)
    assert ipivo[250] == 260
    LU, ipiv, _ = _lu16_gpu(A16, 128, 1, 0)
    assert np.array_equal(ipiv, ipivo) and np.array_equal(LU, LUo)


@pytest.mark.parametrize("row", [2, 200])
def test_lu16_fast_path_compares_unrounded_pivot(row):
    """Partial pivoting compares binary32 values before the pivot row is
    rounded to binary16.  After the first elimination step column 1 holds
    1 + 1.25 * 2^-11 on the diagonal (binary16 rounds it up to 1 + 2^-10) and
    1 + 1.5 * 2^-11 in `row` (inside the diagonal block, or below it): the
    larger one must become the pivot, so the fast path has to notice that the
    diagonal loses although it wins after rounding."""
    N = 300
    rng = np.random.default_rng(5)
    B = 4.0 * np.eye(N) + rng.uniform(-0.01, 0.01, (N, N))
    B[:, 0] = rng.uniform(-0.01, 0.01, N)
    B[:, 1] = rng.uniform(-0.01, 0.01, N)
    B[0, 0] = B[0, 1] = 1.0
    B[1, 0], B[1, 1] = -1.25 * 2.0 ** -11, 1.0
    B[row, 0], B[row, 1] = -1.5 * 2.0 ** -11, 1.0
    A16 = O.fl16(B)
    LUo, ipivo, _, _ = O.lu16_dev(A16, 128)
    assert ipivo[1] == row
    LU, ipiv, _ = _lu16_gpu(A16, 128, 1, 0)
    assert np.array_equal(ipiv, ipivo) and np.array_equal(LU, LUo)


def test_lu16_random_pivoting_valid():
    """Gaussian matrices (near-ties possible): pivots are a valid partial
    pivoting sequence and P A = L U to binary16 accuracy."""
    N = 300
    A16 = O.fl16(W.random_matrix(N, 77))
    LU, ipiv, info = _lu16_gpu(A16, 64, 1)
    assert info == 0
    L = np.tril(LU, -1) + np.eye(N)
    U = np.triu(LU)
    PA = A16.copy()
    for k, p in enumerate(ipiv):
        PA[[k, p]] = PA[[p, k]]
    assert np.max(np.abs(L)) <= 1.0
    rel = np.linalg.norm(PA - L @ U) / np.linalg.norm(A16)
    assert rel <= 0.05 * np.sqrt(N) * 2.0 ** -11 * 10


@pytest.mark.parametrize("N", [12000, 20480])
@pytest.mark.parametrize("nb", [128, 256])
def test_lu16_wide_offdiag_launches_bitwise(N, nb):
    """Large panels: at N = 12000 the early panels' off-diagonal solves exceed
    one wave of 128-row CTAs, so the two-launch path (path 2) takes 256 rows
    per CTA; at N = 20480 the early panels also have more rows than one
    streaming launch holds at once, so the streaming path (path 0) streams
    as many as fit and solves the rest in a following off-diagonal launch.
    Both paths give the bits of each other (every row and column is solved
    by one thread in the same order), one level (nb 128) and two levels
    (nb 256, inner panels on the single-precision shadow), with the SIMT
    update.  The Jacobian of eq. (3.2) at x = 1 + sin^2, formed on the GPU."""
    c = 0.99
    ld = ((N + 63) // 64) * 64
    x = torch.as_tensor(1.0 + 0.5 * np.sin(np.arange(N) * 0.37) ** 2, device=dev())
    F = torch.empty(N, device=dev(), dtype=torch.float64)
    r = torch.empty(N, device=dev(), dtype=torch.float64)
    nrm = torch.empty(1, device=dev(), dtype=torch.float64)
    nl.k_residual(N, c, x, F, r, nrm)
    J32 = torch.empty((N, ld), device=dev(), dtype=torch.float32)
    J16 = torch.zeros((N, ld), device=dev(), dtype=torch.float16)
    nl.k_jacobian(N, c, r, J32, ld, J16, ld)
    del J32
    out = []
    for path in (0, 2):
        A = J16.clone()
        ip = torch.empty(N, device=dev(), dtype=torch.int32)
        info = nl.lu16(N, A, ld, ip, nb=nb, gemm=1, path=path)
        assert info == 0
        assert np.array_equal(ip.cpu().numpy(), np.arange(N))
        out.append(A.cpu().numpy()[:, :N])
        del A
    assert np.array_equal(out[0].view(np.uint16), out[1].view(np.uint16))


@pytest.mark.parametrize("N", [12000, 20480])
def test_lu16_lookahead_wide_panels_bitwise(N):
    """Look-ahead with the tcgen05 update on panels wider than one streaming
    launch (the rows that do not fit go to a following off-diagonal launch):
    the factors of nl_lu16 path 4 are the bits of path 0.  The Jacobian of
    eq. (3.2) at x = 1 + sin^2, formed on the GPU."""
    c = 0.99
    ld = ((N + 63) // 64) * 64
    x = torch.as_tensor(1.0 + 0.5 * np.sin(np.arange(N) * 0.37) ** 2, device=dev())
    F = torch.empty(N, device=dev(), dtype=torch.float64)
    r = torch.empty(N, device=dev(), dtype=torch.float64)
    nrm = torch.empty(1, device=dev(), dtype=torch.float64)
    nl.k_residual(N, c, x, F, r, nrm)
    J32 = torch.empty((N, ld), device=dev(), dtype=torch.float32)
    J16 = torch.zeros((N, ld), device=dev(), dtype=torch.float16)
    nl.k_jacobian(N, c, r, J32, ld, J16, ld)
    del J32
    out = []
    for path in (0, 4):
        A = J16.clone()
        ip = torch.empty(N, device=dev(), dtype=torch.int32)
        assert nl.lu16(N, A, ld, ip, nb=128, gemm=2, path=path) == 0
        assert np.array_equal(ip.cpu().numpy(), np.arange(N))
        out.append(A.cpu().numpy()[:, :N])
        del A
    assert np.array_equal(out[0].view(np.uint16), out[1].view(np.uint16))


@pytest.mark.parametrize("N,nb", [(200, 64), (517, 128), (1024, 128), (777, 64)])
def test_lu16_tensor_core_close_to_oracle(N, nb):
    """tcgen05 trailing update: same pivots, factors within binary16
    rounding of the oracle (the tensor cores sum the K products in their own
    order, so a few entries round to the neighbouring binary16 value)."""
    A, _ = W.pivot_forcing_matrix(N, 2000 + N)
    A16 = O.fl16(A)
    LU, ipiv, info = _lu16_gpu(A16, nb, 2)
    LUo, ipivo, _, _ = O.lu16_dev(A16, nb)
    assert info == 0 and np.array_equal(ipiv, ipivo)
    scale = np.maximum(np.abs(LUo), np.abs(np.diag(LUo)).max() * 2.0 ** -11)
    assert np.max(np.abs(LU - LUo) / scale) <= 8 * 2.0 ** -11
    assert np.mean(LU == LUo) >= 0.95


def _jacobian16(N, c):
    return O.fl16(O.jacobian(N, c, np.ones(N)).astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("N,nb,path", [(1000, 256, 0), (1400, 512, 0), (2100, 384, 0), (1100, 256, 2), (600, 512, 0)])
def test_lu16_two_level_simt_bit_exact(N, nb, path):
    """Two-level factorisation (outer block nb > 128, inner panels of 128
    carried in single precision, one update of depth nb per outer block) with
    the SIMT update: operation for operation the oracle's elimination with
    rounding period nb, on the paper's Jacobian (no interchanges), with the
    streaming panel (path 0) and with the two launches per inner panel (2).
    N = 600 with nb = 512 leaves an outer block of 88 columns."""
    J16 = _jacobian16(N, 0.99)
    LUo, ipivo, _, _ = O.lu16_dev(J16, nb)
    assert np.array_equal(ipivo, np.arange(N))
    LU, ipiv, info = _lu16_gpu(J16, nb, 1, path)
    assert info == 0 and np.array_equal(ipiv, ipivo)
    assert np.array_equal(LU, LUo)


@pytest.mark.parametrize("N,nb", [(1000, 256), (2300, 512), (4096, 512)])
def test_lu16_two_level_tensor_core_close_to_oracle(N, nb):
    """The same with the tcgen05 update of depth nb (the persistent kernel
    streaming K through its operand ring): same pivots, factors within
    binary16 rounding of the oracle with rounding period nb, and far more
    accurate than the oracle's period-128 factors are from them."""
    J16 = _jacobian16(N, 0.9999)
    LUo, ipivo, _, _ = O.lu16_dev(J16, nb)
    LU, ipiv, info = _lu16_gpu(J16, nb, 2)
    assert info == 0 and np.array_equal(ipiv, ipivo)
    scale = np.maximum(np.abs(LUo), np.abs(np.diag(LUo)).max() * 2.0 ** -11)
    assert np.max(np.abs(LU - LUo) / scale) <= 8 * 2.0 ** -11
    assert np.mean(LU == LUo) >= 0.95


@pytest.mark.parametrize("N,nb", [(300, 128), (777, 64), (1000, 128), (2049, 64), (4100, 128)])
def test_lu16_lookahead_bitwise(N, nb):
    """Look-ahead (nl_lu16 path 4): after each panel only the trailing
    matrix's first tile row and column are updated on the caller's stream,
    the rest on a second stream in the shadow of the next panel.  The same
    tcgen05 tiles, so the factors are the bits of the one-update path (0),
    which is itself within binary16 rounding of the oracle; N = 300 ends with
    a trailing matrix of one tile strip (no side-stream update), N = 4100
    with a ragged 4-column panel."""
    J16 = _jacobian16(N, 0.99)
    LU0, ip0, info0 = _lu16_gpu(J16, nb, 2, 0)
    LU4, ip4, info4 = _lu16_gpu(J16, nb, 2, 4)
    assert info0 == info4 == 0 and np.array_equal(ip0, ip4) and np.array_equal(ip4, np.arange(N))
    assert np.array_equal(LU0.view(np.uint64), LU4.view(np.uint64))
    if N <= 2049:
        LUo, _, _, _ = O.lu16_dev(J16, nb)
        scale = np.maximum(np.abs(LUo), np.abs(np.diag(LUo)).max() * 2.0 ** -11)
        assert np.max(np.abs(LU4 - LUo) / scale) <= 8 * 2.0 ** -11
        assert np.mean(LU4 == LUo) >= 0.95


def test_lu16_lookahead_falls_back_to_interchanges():
    """A matrix that needs row interchanges: the look-ahead fast path is
    abandoned (its side-stream updates see the flag) and the interchanging
    path gives the same factors as without look-ahead."""
    N = 700
    A, _ = W.pivot_forcing_matrix(N, 3101)
    A16 = O.fl16(A)
    LU0, ip0, info0 = _lu16_gpu(A16, 128, 2, 0)
    LU4, ip4, info4 = _lu16_gpu(A16, 128, 2, 4)
    assert info0 == info4 == 0 and not np.array_equal(ip0, np.arange(N))
    assert np.array_equal(ip0, ip4) and np.array_equal(LU0.view(np.uint64), LU4.view(np.uint64))


def test_lu16_two_level_falls_back_to_interchanges():
    """A matrix that needs row interchanges: the two-level fast path detects
    it and the factorisation is redone by the interchanging path with outer
    block 128, equal to the oracle's period-128 elimination."""
    N = 700
    A, _ = W.pivot_forcing_matrix(N, 3100)
    A16 = O.fl16(A)
    LU, ipiv, info = _lu16_gpu(A16, 512, 1, 0)
    LUo, ipivo, infoo, _ = O.lu16_dev(A16, 128)
    assert info == infoo == 0 and np.array_equal(ipiv, ipivo) and np.array_equal(LU, LUo)


def test_lu16_zero_column_reports_info():
    N = 40
    A, _ = W.pivot_forcing_matrix(N, 5)
    A[:, 17] = 0.0
    A16 = O.fl16(A)
    _, _, info = _lu16_gpu(A16, 16, 1)
    _, _, infoo, _ = O.lu16_dev(A16, 16)
    assert info == infoo == 18


# ------------------------------------------------------------ GEMM update --

@pytest.mark.parametrize("M,Nc,K", [(128, 128, 128), (300, 200, 128), (129, 1000, 88), (1, 5, 16), (2000, 2100, 128),
                                    (257, 130, 64), (77, 3000, 1), (4000, 384, 128)])
def test_update32_tensor_core(M, Nc, K):
    """nl_k_update32 (the two-level LU's inner update on the tensor cores):
    C <- C - A B for binary32 C and binary16-valued A, B.  The products are
    exact, so the result is the exact C - A B up to the tensor cores' binary32
    summation and one rounding: within (K + 2) 2^-23 (|C| + |A| |B|) of the
    double-precision value.  Entries outside M x Nc (the leading dimensions'
    padding) are untouched, and a second call gives the same bits."""
    g = np.random.default_rng(M * 13 + Nc + K)
    A = g.uniform(-1, 1, (M, K)).astype(np.float16).astype(np.float32)
    B = g.uniform(-1, 1, (K, Nc)).astype(np.float16).astype(np.float32)
    C = g.uniform(-4, 4, (M, Nc)).astype(np.float32)
    lda, ldb, ldc = K + 5, Nc + 3, Nc + 7  # odd strides: the scalar load paths
    Ad = torch.full((M, lda), 7.0, device=dev(), dtype=torch.float32)
    Bd = torch.full((K, ldb), 7.0, device=dev(), dtype=torch.float32)
    Cd = torch.full((M + 1, ldc), -3.0, device=dev(), dtype=torch.float32)
    Ad[:, :K] = T(A)
    Bd[:, :Nc] = T(B)
    Cd[:M, :Nc] = T(C)
    C0 = Cd.clone()
    nl.k_update32(M, Nc, K, Ad, lda, Bd, ldb, Cd, ldc)
    out = Cd.cpu().numpy()
    exact = C.astype(np.float64) - A.astype(np.float64) @ B.astype(np.float64)
    bound = (K + 2) * 2.0 ** -23 * (np.abs(C) + np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64))
    assert np.all(np.abs(out[:M, :Nc] - exact) <= bound)
    assert np.array_equal(out[:M, Nc:], C0.cpu().numpy()[:M, Nc:]) and np.all(out[M] == -3.0)
    Cd2 = C0.clone()
    nl.k_update32(M, Nc, K, Ad, lda, Bd, ldb, Cd2, ldc)
    assert np.array_equal(Cd2.cpu().numpy(), out)


def test_update32_aligned_strides_match_scalar_paths():
    """The vector (16-byte) load and store paths give the bits of the scalar
    ones (the same values in the same order)."""
    M, Nc, K = 640, 512, 128
    g = np.random.default_rng(5)
    A = g.uniform(-1, 1, (M, K)).astype(np.float16).astype(np.float32)
    B = g.uniform(-1, 1, (K, Nc)).astype(np.float16).astype(np.float32)
    C = g.uniform(-4, 4, (M, Nc)).astype(np.float32)
    outs = []
    for pad in (0, 1):
        Ad = torch.zeros((M, K + pad), device=dev(), dtype=torch.float32)
        Bd = torch.zeros((K, Nc + pad), device=dev(), dtype=torch.float32)
        Cd = torch.zeros((M, Nc + pad), device=dev(), dtype=torch.float32)
        Ad[:, :K], Bd[:, :Nc], Cd[:, :Nc] = T(A), T(B), T(C)
        nl.k_update32(M, Nc, K, Ad, K + pad, Bd, Nc + pad, Cd, Nc + pad)
        outs.append(Cd.cpu().numpy()[:, :Nc])
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("M,Nc,K", [(64, 64, 64), (300, 200, 128), (129, 1000, 256), (1, 5, 64), (2000, 2100, 128),
                                    (3000, 2900, 64), (700, 900, 512), (300, 129, 1024), (1100, 1300, 384)])
def test_gemm16_update(M, Nc, K):
    """C <- fl16(C - A B): SIMT bitwise the sequential single-precision sums;
    tcgen05 within the binary16 rounding of the exact result.  The persistent
    kernel streams K through its four-slot operand ring (any multiple of 64 up
    to 1024: the LU's outer block); up to K = 256 it equals the one-tile-per-CTA
    kernel bit for bit (the same MMAs in the same order)."""
    g = np.random.default_rng(M * 7 + Nc)
    A = g.uniform(-1, 1, (M, K)).astype(np.float16)
    B = g.uniform(-1, 1, (K, Nc)).astype(np.float16)
    C = g.uniform(-4, 4, (M, Nc)).astype(np.float16)
    ld = lambda n: ((n + 63) // 64) * 64
    res = {}
    for gemm in ((1, 2, 3) if K <= 256 else (1, 2)):
        Ad = torch.zeros((M, ld(K)), device=dev(), dtype=torch.float16)
        Bd = torch.zeros((K, ld(Nc)), device=dev(), dtype=torch.float16)
        Cd = torch.zeros((M, ld(Nc)), device=dev(), dtype=torch.float16)
        Ad[:, :K] = T(A)
        Bd[:, :Nc] = T(B)
        Cd[:, :Nc] = T(C)
        nl.k_gemm16_update(M, Nc, K, Ad, ld(K), Bd, ld(Nc), Cd, ld(Nc), gemm=gemm)
        res[gemm] = Cd.cpu().numpy()[:, :Nc]
    # SIMT: sequential single-precision fused multiply-adds (the product of two
    # binary16 numbers is exact in single, so this is a - a_k b_k rounded)
    acc = C.astype(np.float32)
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    for k in range(K):
        acc = (acc - A32[:, k:k + 1] * B32[k:k + 1, :]).astype(np.float32)
    assert np.array_equal(res[1], acc.astype(np.float16))
    exact = C.astype(np.float64) - A.astype(np.float64) @ B.astype(np.float64)
    tol = np.abs(exact) * 2.0 ** -10 + K * 2.0 ** -20 * 4
    assert np.all(np.abs(res[2].astype(np.float64) - exact) <= tol)
    # the persistent pipelined kernel and the one-tile-per-CTA kernel issue the
    # same MMAs and the same epilogue: bitwise the same
    if K <= 256:
        assert np.array_equal(res[2], res[3])


# -------------------------------------------------------------- K4 / K7 --

@pytest.mark.parametrize("N", [1, 5, 64, 100, 333, 1000])
def test_lusolve16_matches_oracle_fly(N):
    A, _ = W.pivot_forcing_matrix(N, 3000 + N)
    A16 = O.fl16(A)
    LUo, ipivo, _, _ = O.lu16_dev(A16, 64)
    b = W.random_vector(N, 4000 + N).astype(np.float32)
    ref = O.lusolve_fly(LUo, ipivo, b).astype(np.float64)
    ld = ((N + 63) // 64) * 64
    LUd = torch.zeros((N, ld), device=dev(), dtype=torch.float16)
    LUd[:, :N] = T(LUo.astype(np.float16))
    bd = T(b)
    nl.lusolve16(N, LUd, ld, T(ipivo.astype(np.int32)), bd)
    got = bd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 2e-5 * np.linalg.norm(ref)


def synthetic_factors(N, seed):
    """Binary16 factors with a known-stable solve: unit lower L and upper U
    whose off-diagonal entries are uniform in (-2/N, 2/N) (so a skipped or
    misplaced 128-column tile changes x by far more than the tolerance),
    U's diagonal of magnitude in [1, 2] with random signs, and a random
    valid pivot sequence ipiv[k] in [k, N)."""
    rng = np.random.default_rng(seed)
    LU = rng.uniform(-2.0 / N, 2.0 / N, size=(N, N))
    d = rng.uniform(1.0, 2.0, size=N) * rng.choice([-1.0, 1.0], size=N)
    LU[np.arange(N), np.arange(N)] = d
    LU = LU.astype(np.float16).astype(np.float64)
    ipiv = np.array([rng.integers(k, N) for k in range(N)], dtype=np.int32)
    return LU, ipiv


@pytest.mark.parametrize("N", [127, 128, 2049, 4096, 4097, 9000])
def test_lusolve16_synthetic_factors(N):
    """Both triangles over many 128-row blocks, with ragged last blocks and
    more blocks than CTAs in one cluster (each CTA owns several blocks)."""
    LUo, ipivo = synthetic_factors(N, 5000 + N)
    b = W.random_vector(N, 6000 + N).astype(np.float32)
    ref = O.lusolve_fly(LUo, ipivo, b).astype(np.float64)
    ld = ((N + 63) // 64) * 64
    LUd = torch.zeros((N, ld), device=dev(), dtype=torch.float16)
    LUd[:, :N] = T(LUo.astype(np.float16))
    bd = T(b)
    nl.lusolve16(N, LUd, ld, T(ipivo), bd)
    got = bd.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 * np.max(np.abs(ref)))


@pytest.mark.parametrize("N,kind", [(1, "rand"), (2, "rand"), (7, "rand"), (100, "rand"), (333, "rand"),
                                    (600, "piv"), (50, "sing"), (1000, "rand")])
def test_lu16_binary16_arithmetic_bit_exact(N, kind):
    """nl_lu16 path 3: every operation rounded to binary16 (the arithmetic of
    the F16 column), partial pivoting with whole-row swaps: pivots, factors
    and info bitwise the oracle's binary16 LU.  A Gaussian matrix swaps rows
    at most steps; "sing" has a zero column (info = 11, that step skipped)."""
    if kind == "piv":
        A = W.pivot_forcing_matrix(N, 12000 + N)[0]
    else:
        A = W.random_matrix(N, 12000 + N)
        if kind == "sing":
            A[:, 10] = 0.0
    A16 = O.fl16(A)
    LUo, ipivo, infoo, ovfo = O.lu16(A16)
    assert not ovfo
    ld = ((N + 63) // 64) * 64
    Ad = torch.zeros((N, ld), device=dev(), dtype=torch.float16)
    Ad[:, :N] = T(A16.astype(np.float16))
    ipiv = torch.empty(N, device=dev(), dtype=torch.int32)
    info = nl.lu16(N, Ad, ld, ipiv, path=3)
    assert info == infoo == (11 if kind == "sing" else 0)
    assert np.array_equal(ipiv.cpu().numpy(), ipivo)
    assert np.array_equal(Ad.cpu().numpy()[:, :N].astype(np.float64), LUo)


# ------------------------------------------------- F32 / F16 columns --

@pytest.mark.parametrize("N,nb", [(1, 16), (50, 16), (200, 64), (301, 128), (1000, 128)])
def test_lu32_and_solve_match_oracle(N, nb):
    """Single-precision LU with interchanges (the F32 column, Section 1.3).
    A pivot-forcing matrix has one pivot sequence with a wide gap, so ipiv
    must equal the oracle's exactly; the factors differ from the oracle's
    only by the order and fusing of single-precision operations (measured
    ~1.5e-6 of max|LU| at N = 1000; a misplaced term changes them by O(1)).
    The solve is checked against the double solve of the same system."""
    A, _ = W.pivot_forcing_matrix(N, 7000 + N)
    A32 = A.astype(np.float32)
    ld = ((N + 63) // 64) * 64
    Ad = torch.zeros((N, ld), device=dev(), dtype=torch.float32)
    Ad[:, :N] = T(A32)
    ipiv = torch.empty(N, device=dev(), dtype=torch.int32)
    info = nl.lu32(N, Ad, ld, ipiv, nb=nb)
    LUo, ipivo, infoo = O.lu32(A32)
    assert info == infoo == 0
    assert np.array_equal(ipiv.cpu().numpy(), ipivo)
    LU = Ad.cpu().numpy()[:, :N].astype(np.float64)
    scale = np.max(np.abs(LUo))
    assert np.max(np.abs(LU - LUo)) <= 2e-5 * scale
    # partial pivoting: every multiplier at most 1 in magnitude
    assert np.max(np.abs(np.tril(LU, -1)), initial=0.0) <= 1.0
    b = W.random_vector(N, 8000 + N).astype(np.float32)
    bd = T(b)
    nl.lusolve32(N, Ad, ld, ipiv, bd)
    LU64, ip64, _ = O.lu64(A32.astype(np.float64))
    ref = O.lusolve64(LU64, ip64, b.astype(np.float64))
    got = bd.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [127, 128, 2049, 4097, 9000])
def test_lusolve32_synthetic_factors(N):
    """The single-precision blocked solve over many 64-row blocks (more than
    the cooperative grid's CTAs at 9000), ragged last blocks, against the
    oracle's sequential single-precision solve."""
    LUo, ipivo = synthetic_factors(N, 9000 + N)
    b = W.random_vector(N, 9500 + N).astype(np.float32)
    ref = O.lusolve32(LUo.astype(np.float32), ipivo, b).astype(np.float64)
    ld = ((N + 63) // 64) * 64
    LUd = torch.zeros((N, ld), device=dev(), dtype=torch.float32)
    LUd[:, :N] = T(LUo.astype(np.float32))
    bd = T(b)
    nl.lusolve32(N, LUd, ld, T(ipivo), bd)
    got = bd.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 * np.max(np.abs(ref)))


@pytest.mark.parametrize("N,kind,ld_mode", [(1, "syn", 64), (5, "syn", 64), (127, "syn", 64), (1000, "syn", 64),
                                            (2049, "syn", 64), (3000, "syn", 64), (4096, "syn", 64),
                                            (333, "lu16", 64), (1001, "syn", 1), (4097, "syn", 64),
                                            (9000, "syn", 64)])
def test_lusolve16h_bit_exact(N, kind, ld_mode):
    """Both triangular solves in binary16 arithmetic (the F16 step and the
    correction of eq. (2.19)): every product and difference rounded to
    binary16 in the oracle's order, so the result is bitwise the oracle's.
    N <= 4096 with ld a multiple of 8 takes the register-pipelined sweep
    (1, 2 and 4 rows per thread); ld = N odd (1001) and N > 4096 the scalar
    one."""
    if kind == "syn":
        LUo, ipivo = synthetic_factors(N, 10000 + N)
    else:
        A, _ = W.pivot_forcing_matrix(N, 10500 + N)
        LUo, ipivo, info, ovf = O.lu16_dev(O.fl16(A), 64)
        assert info == 0 and not ovf
    b16 = O.fl16(W.random_vector(N, 11000 + N) / 4)
    ref = O.lusolve16(LUo, ipivo, b16)
    ld = ((N + ld_mode - 1) // ld_mode) * ld_mode
    LUd = torch.zeros((N, ld), device=dev(), dtype=torch.float16)
    LUd[:, :N] = T(LUo.astype(np.float16))
    bd = T(b16.astype(np.float16))
    nl.lusolve16h(N, LUd, ld, T(ipivo.astype(np.int32)), bd)
    got = bd.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(ref))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("N,nb,diag", [(1, 16, False), (50, 16, False), (200, 64, False), (301, 64, False),
                                        (301, 64, True), (500, 128, True)])
def test_lu64_and_solve_match_oracle(N, nb, diag):
    A = W.random_matrix(N, 5000 + N)
    if diag:  # diagonally dominant by rows and columns: no interchanges (fast path)
        A += np.diag(np.abs(A).sum(axis=0) + np.abs(A).sum(axis=1))
    ld = ((N + 63) // 64) * 64
    Ad = torch.zeros((N, ld), device=dev(), dtype=torch.float64)
    Ad[:, :N] = T(A)
    ipiv = torch.empty(N, device=dev(), dtype=torch.int32)
    info = nl.lu64(N, Ad, ld, ipiv, nb=nb)
    LUo, ipivo, infoo = O.lu64(A)
    assert info == infoo == 0
    assert np.array_equal(ipiv.cpu().numpy(), ipivo)
    LU = Ad.cpu().numpy()[:, :N]
    assert np.max(np.abs(LU - LUo)) <= 1e-11 * max(1.0, np.max(np.abs(LUo)))
    b = W.random_vector(N, 6000 + N)
    bd = T(b)
    nl.lusolve64(N, Ad, ld, ipiv, bd)
    ref = O.lusolve64(LUo, ipivo, b)
    assert np.linalg.norm(bd.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref) * max(1, np.linalg.cond(A) / 1e3)


# ------------------------------------------------------------ K5 / IR / GMRES

@pytest.mark.parametrize("N", [3, 256, 1001])
def test_gemv_residual(N):
    g = np.random.default_rng(N)
    A = g.standard_normal((N, N)).astype(np.float32)
    u = g.standard_normal(N).astype(np.float32)
    b = g.standard_normal(N).astype(np.float32)
    ld = ((N + 63) // 64) * 64
    Ad = torch.zeros((N, ld), device=dev(), dtype=torch.float32)
    Ad[:, :N] = T(A)
    ud = torch.zeros(ld, device=dev(), dtype=torch.float32)
    ud[:N] = T(u)
    r = torch.empty(N, device=dev(), dtype=torch.float32)
    rn = torch.empty(1, device=dev(), dtype=torch.float64)
    nl.k_gemv_residual(N, Ad, ld, T(b), ud, r, rn)
    exact = b.astype(np.float64) - A.astype(np.float64) @ u.astype(np.float64)
    # compensated accumulation: the single result is within one rounding of
    # the exact residual plus a second-order term
    bound = 2.0 ** -24 * np.abs(exact) + 4 * N * 2.0 ** -46 * (np.abs(A).astype(np.float64) @ np.abs(u) + np.abs(b))
    got = r.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - exact) <= bound)
    # and it equals the oracle's residual (double accumulation, one rounding)
    # except where the two round to neighbouring single values
    ref = exact.astype(np.float32).astype(np.float64)
    assert np.mean(got == ref) >= 0.99
    assert abs(rn.item() - np.linalg.norm(got)) <= 1e-12 * np.linalg.norm(got)


@pytest.mark.parametrize("solver", [0, 2])
@pytest.mark.parametrize("N,c", [(300, 0.9), (1000, 0.99)])
def test_linsolve16_matches_oracle(solver, N, c):
    """IR and GMRES-IR with identical inputs (J32, binary16 factors, b):
    same outcome, iteration counts within one, solutions within eta."""
    x = np.ones(N)
    J = O.jacobian(N, c, x)
    J32 = J.astype(np.float32)
    LUo, ipivo, _, _ = O.lu16_dev(O.fl16(J32.astype(np.float64)), 128)
    F = O.F(N, c, x)
    b = (-F / np.linalg.norm(F)).astype(np.float32)
    # eta above the single-precision noise floor of the preconditioned
    # iteration (about kappa * u_s), where the outcome is not decided by rounding
    eta = 1e-5
    uo, sto = O.linsolve(J32, LUo, ipivo, b, solver=solver, eta=eta, maxit=20)
    ld = ((N + 63) // 64) * 64
    Jd = torch.zeros((N, ld), device=dev(), dtype=torch.float32)
    Jd[:, :N] = T(J32)
    LUd = torch.zeros((N, ld), device=dev(), dtype=torch.float16)
    LUd[:, :N] = T(LUo.astype(np.float16))
    ud = torch.zeros(ld, device=dev(), dtype=torch.float32)
    st = nl.linsolve16(N, Jd, ld, LUd, ld, T(ipivo.astype(np.int32)), T(b), ud, eta=eta, maxit=20, solver=solver)
    assert st["converged"] == sto["converged"] == 1
    assert abs(st["iters"] - sto["iters"]) <= 1 and st["failed"] == sto["failed"] == 0
    got = ud.cpu().numpy()[:N].astype(np.float64)
    assert np.linalg.norm(got - uo) <= 10 * eta * np.linalg.norm(uo) * np.linalg.cond(J32.astype(np.float64))
    assert st["relres"] <= eta


def test_multiplier_rounding_exact_vs_ieee():
    """The LU forms l = fl16(a / u) from a correctly rounded reciprocal; it
    must equal fl16 of the IEEE single-precision quotient for every input,
    including quotients within a few single-precision units of a binary16
    rounding boundary (the cases its exactness test sends to the division)."""
    g = np.random.default_rng(12)
    n = 1 << 20
    # divisors: binary16 values (the rounded pivots), both signs, normal and subnormal
    u16 = g.integers(1, 0x7C00, size=n).astype(np.uint16) | (g.integers(0, 2, size=n).astype(np.uint16) << 15)
    u = u16.view(np.float16).astype(np.float32)
    a = (g.uniform(-1.0, 1.0, size=n) * np.abs(u)).astype(np.float32)
    # a quarter of the numerators aimed at binary16 midpoints: a ~ m u, nudged by a few units
    k = n // 4
    h = g.integers(0x0000, 0x7BFF, size=k).astype(np.uint16)
    h[: k // 4] = g.integers(0x0000, 0x0400, size=k // 4)  # binary16 subnormal boundaries, 2^-25 included
    lo = h.view(np.float16).astype(np.float64)
    hi = (h + 1).view(np.float16).astype(np.float64)
    m = (lo + hi) / 2.0 * np.where(g.integers(0, 2, size=k) == 1, 1.0, -1.0)
    aa = (m * u[:k].astype(np.float64)).astype(np.float32)
    nudge = g.integers(-6, 7, size=k)
    a[:k] = aa + nudge.astype(np.float32) * np.spacing(aa)
    a[:16] = np.array([0.0, -0.0, 1.0, -1.0] * 4, dtype=np.float32)
    # exact binary16 midpoints times u (ties at both precisions) and tiny quotients
    a[16:32] = (np.float32(2.0 ** -25) * u[16:32]).astype(np.float32)
    a[32:48] = (np.float32(0.5 * (1.0 + (1.0 - 2.0 ** -11))) * u[32:48]).astype(np.float32)
    a[48:64] = (np.float32(2.0 ** -30) * u[48:64]).astype(np.float32)
    ref32 = (a / u).astype(np.float32)  # IEEE single division (numpy)
    ref = O.f16_bits_from_f32(ref32)
    out = torch.empty(n, device=dev(), dtype=torch.float32)
    nl.k_div_round16(n, T(a), T(u), out)
    got = O.f16_bits_from_f32(out.cpu().numpy())
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, (bad[:5], a[bad[:5]], u[bad[:5]])
