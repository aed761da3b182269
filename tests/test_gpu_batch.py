"""Batched path (grouped LU, grouped triangular solves, graph-captured
Newton over many instances) against the single-instance CUDA path and the
CPU oracle, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16051_gb300 import nl
from paper_2307_16051_gb300 import workloads as W
from tests.conftest import newton_counts_agree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def rel_inf(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def jacobian16(N, c, seed):
    """binary16 Jacobian of eq. (3.2) at a random positive iterate (oracle J,
    rounded to single then to binary16 as the method does)."""
    g = np.random.default_rng(seed)
    x = 1.0 + g.uniform(0.0, 1.0, N)
    return O.fl16(O.jacobian(N, c, x).astype(np.float32).astype(np.float64))


def padded16(A16, ld):
    N = A16.shape[0]
    a = np.zeros((N, ld), dtype=np.float16)
    a[:, :N] = A16.astype(np.float16)
    return torch.as_tensor(a, device=dev())


def lu_single(A16, ld, nb, gemm):
    N = A16.shape[0]
    A = padded16(A16, ld)
    ip = torch.empty(N, dtype=torch.int32, device=dev())
    nl.lu16(N, A, ld, ip, nb=nb, gemm=gemm, path=0)
    return A.cpu().numpy()[:, :N].astype(np.float64), ip.cpu().numpy()


def lu_grouped(mats, nb, gemm, fp64=False):
    Ns, As, lds, ips = [], [], [], []
    for M in mats:
        N = M.shape[0]
        ld = ((N + 63) // 64) * 64
        if fp64:
            a = np.zeros((N, ld))
            a[:, :N] = M
            A = torch.as_tensor(a, device=dev())
        else:
            A = padded16(M, ld)
        Ns.append(N)
        As.append(A)
        lds.append(ld)
        ips.append(torch.full((N,), -1, dtype=torch.int32, device=dev()))
    flags = nl.lu_grouped(Ns, As, lds, ips, fp64=fp64, nb=nb, gemm=gemm)
    torch.cuda.synchronize()
    out = [(A.cpu().numpy()[:, :n].astype(np.float64), p.cpu().numpy()) for A, p, n in zip(As, ips, Ns)]
    return out, flags


SIZES = [1, 17, 64, 130, 300, 513, 1000]


@pytest.mark.parametrize("nb,gemm", [(128, 2), (64, 2), (64, 1), (32, 1)])
def test_lu_grouped_identical_to_single(nb, gemm):
    """The grouped launch runs the single-matrix kernels on every matrix of
    the group: factors and pivots are bit-for-bit those of nl_lu16."""
    mats = [jacobian16(N, 0.5 + 0.049 * k, 100 + k) for k, N in enumerate(SIZES)]
    out, flags = lu_grouped(mats, nb, gemm)
    assert not flags.any()
    for M, (LU, ip) in zip(mats, out):
        N = M.shape[0]
        LUs, ips = lu_single(M, ((N + 63) // 64) * 64, nb, gemm)
        assert np.array_equal(ip, np.arange(N))
        assert np.array_equal(ips, ip)
        assert np.array_equal(LU, LUs), N


@pytest.mark.parametrize("nb", [128, 48])
def test_lu_grouped_simt_bit_exact_vs_oracle(nb):
    """With the SIMT update the grouped factors equal the oracle's binary16
    storage / binary32 arithmetic elimination (rounding period nb) exactly."""
    mats = [jacobian16(N, 0.99, 7 + N) for N in (33, 200, 401)]
    out, flags = lu_grouped(mats, nb, 1)
    assert not flags.any()
    for M, (LU, ip) in zip(mats, out):
        LUo, ipo, info, ovf = O.lu16_dev(M, nb)
        assert info == 0 and not ovf
        assert np.array_equal(ip, ipo)
        assert np.array_equal(LU, LUo)


def test_lu_grouped_flags_matrices_that_need_interchanges():
    """A matrix on which partial pivoting swaps rows is flagged (and left to
    the interchanging path); its neighbours in the group are unaffected."""
    P, _ = W.pivot_forcing_matrix(150, 3)
    mats = [jacobian16(90, 0.9, 1), O.fl16(P), jacobian16(260, 0.99, 2), O.fl16(W.pivot_forcing_matrix(70, 4)[0])]
    out, flags = lu_grouped(mats, 64, 2)
    assert list(flags) == [0, 1, 0, 1]
    for k in (0, 2):
        N = mats[k].shape[0]
        LUs, ips = lu_single(mats[k], ((N + 63) // 64) * 64, 64, 2)
        assert np.array_equal(out[k][0], LUs) and np.array_equal(out[k][1], ips)


def test_lu_grouped_fp64_matches_oracle():
    """Grouped double LU (the FP64 baseline's factorisation): P A = L U equal
    to the oracle's partial-pivoting elimination to rounding, no interchanges
    on the H-equation's Jacobians."""
    mats = []
    for k, N in enumerate((5, 64, 129, 333)):
        g = np.random.default_rng(k)
        mats.append(O.jacobian(N, 0.999, 1.0 + g.uniform(0, 1, N)))
    out, flags = lu_grouped(mats, 64, 1, fp64=True)
    assert not flags.any()
    for M, (LU, ip) in zip(mats, out):
        LUo, ipo, info = O.lu64(M)
        assert np.array_equal(ip, ipo)
        assert np.allclose(LU, LUo, rtol=1e-12, atol=1e-14)


def test_lusolve_grouped_matches_oracle():
    """Grouped U^{-1} L^{-1} P b with binary16 factors promoted on the fly
    (eq. (2.16)), including factors with interchanges, against the oracle's
    substitution (single-precision rounding differences only)."""
    systems = []
    for k, N in enumerate((1, 31, 32, 33, 257, 1000, 2048)):
        A16 = jacobian16(N, 0.99, 50 + k) if k % 2 == 0 else O.fl16(W.pivot_forcing_matrix(N, 60 + k)[0])
        LU, ip, info, ovf = O.lu16_dev(A16, 128)
        assert info == 0
        b = np.random.default_rng(k).standard_normal(N).astype(np.float32)
        systems.append((LU, ip, b))
    Ns = [s[0].shape[0] for s in systems]
    lds = [((N + 63) // 64) * 64 for N in Ns]
    LUs = [padded16(s[0], ld) for s, ld in zip(systems, lds)]
    ips = [torch.as_tensor(s[1], device=dev()) for s in systems]
    bs = [torch.as_tensor(s[2], device=dev()) for s in systems]
    nl.lusolve_grouped(Ns, LUs, lds, ips, bs)
    for (LU, ip, b), bd in zip(systems, bs):
        ref = O.lusolve_fly(LU, ip, b).astype(np.float64)
        got = bd.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref)) <= 2e-5 * max(1.0, np.max(np.abs(ref)))


def test_lusolve_grouped_fp64_matches_oracle():
    systems = []
    for k, N in enumerate((3, 100, 700)):
        A = W.random_matrix(N, 5 + k) + N * np.eye(N) * (k % 2)
        LU, ip, info = O.lu64(A)
        b = np.random.default_rng(k).standard_normal(N)
        systems.append((LU, ip, b))
    Ns = [s[0].shape[0] for s in systems]
    LUs = [torch.as_tensor(s[0], device=dev()) for s in systems]
    ips = [torch.as_tensor(s[1], device=dev()) for s in systems]
    bs = [torch.as_tensor(s[2], device=dev()) for s in systems]
    nl.lusolve_grouped(Ns, LUs, Ns, ips, bs, fp64=True)
    for (LU, ip, b), bd in zip(systems, bs):
        ref = O.lusolve64(LU, ip, b)
        assert np.allclose(bd.cpu().numpy(), ref, rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------ batched Newton --

def small_batch(count=24, seed=11, n_lo=17, n_hi=400):
    inst = W.batch_instances(count, seed=seed, n_lo=n_lo, n_hi=n_hi)
    return [n for n, _ in inst], [c for _, c in inst]


def check_instance(st, ro, x, xo, lin=True):
    assert ro["status"] == 0 and st["status"] == nl.NL_OK
    assert newton_counts_agree(st["newton_iters"], ro), (st["newton_iters"], ro["newton_iters"], ro["hist"])
    if lin:
        for a, b in zip(st["lin_iters"], ro["lin_iters"]):
            assert abs(a - b) <= 1, (st["lin_iters"], ro["lin_iters"])
    assert rel_inf(x, xo) <= 1e-10


@pytest.mark.parametrize("nb", [64, 128])
def test_batch_matches_oracle(nb):
    """Every instance of a mixed batch: same Newton count as the oracle's
    IR16-with-GMRES-fallback Newton, linear counts within one, x within 1e-10."""
    Ns, cs = small_batch()
    with nl.Batch(Ns, cs, lu_nb=nb) as B:
        xs, status = B.solve(tol=1e-10, mode="IR16_GMRES")
        info = B.info()
        stats = [B.stats(i) for i in range(len(Ns))]
    assert status == nl.NL_OK and info["converged"] == len(Ns)
    assert info["lu_nb"] == nb and info["newton_rounds"] == max(s["newton_iters"] for s in stats)
    for N, c, x, st in zip(Ns, cs, xs, stats):
        xo, ro = O.newton(N, c, "IR16GM", tol=1e-10, lu_nb=nb)
        check_instance(st, ro, x, xo)


def test_batch_fp64_matches_oracle():
    Ns, cs = small_batch(12, seed=5)
    with nl.Batch(Ns, cs, lu_nb=64) as B:
        xs, status = B.solve(tol=1e-10, mode="FP64LU")
        stats = [B.stats(i) for i in range(len(Ns))]
    assert status == nl.NL_OK
    for N, c, x, st in zip(Ns, cs, xs, stats):
        xo, ro = O.newton(N, c, "FP64LU", tol=1e-10)
        check_instance(st, ro, x, xo, lin=False)


def test_batch_ir_stall_falls_back_to_gmres():
    """One IR correction cannot reach eta = 1e-6: every instance stalls in its
    first step, leaves the batch, and is finished with GMRES-IR; the result
    equals the oracle's fallback rule (which is GMRES-IR from that step on)."""
    Ns, cs = small_batch(8, seed=3, n_hi=200)
    with nl.Batch(Ns, cs, lu_nb=64, ir_maxit=1, eta_j=1e-6) as B:
        xs, status = B.solve(tol=1e-10)
        info = B.info()
        stats = [B.stats(i) for i in range(len(Ns))]
    assert status == nl.NL_OK
    assert info["parked_ir"] == len(Ns) and info["parked_lu"] == 0
    for N, c, x, st in zip(Ns, cs, xs, stats):
        xo, ro = O.newton(N, c, "IR16GM", tol=1e-10, lu_nb=64, ir_maxit=1, eta=1e-6)
        assert ro["lin_failed"][0] == 1 and st["lin_failed"][0] == 1
        check_instance(st, ro, x, xo)


def test_batch_edge_instances_and_repeat():
    """N = 1 (closed form), c = 0 (x0 = ones already solves it: no step), a
    ragged N, and a second solve of the same batch: bitwise the same."""
    Ns, cs = [1, 5, 77, 64, 1], [0.75, 0.0, 0.999, 0.3, 0.0]
    with nl.Batch(Ns, cs, lu_nb=64) as B:
        xs, status = B.solve(tol=1e-10)
        st1 = B.stats(1)
        xs2, _ = B.solve(tol=1e-10)
    assert status == nl.NL_OK
    # the stop at ||F|| <= 1e-10 ||F(x0)|| bounds the error by about kappa 1e-10 ||F(x0)||
    assert abs(xs[0][0] - 2 * (1 - math.sqrt(1 - 0.75)) / 0.75) <= 1e-10
    assert st1["newton_iters"] == 0 and np.all(xs[1] == 1.0)
    for a, b in zip(xs, xs2):
        assert np.array_equal(a, b)
    for N, c, x in zip(Ns[2:4], cs[2:4], xs[2:4]):
        xo, ro = O.newton(N, c, "IR16GM", tol=1e-10, lu_nb=64)
        assert rel_inf(x, xo) <= 1e-10


def test_batch_autotuner_choice_is_used_and_recorded():
    Ns, cs = small_batch(10, seed=9)
    with nl.Batch(Ns, cs) as B:
        info0 = B.info()
        xs, status = B.solve(tol=1e-10)
        info = B.info()
        st = B.stats(0)
    assert status == nl.NL_OK
    cands = {(t[0], t[1]) for t in info0["tune"]}
    assert len(info0["tune"]) >= 2 and (info["lu_nb"], info["trailing_gemm"]) in cands
    best = min(info0["tune"], key=lambda t: t[2])
    assert (best[0], best[1]) == (info["lu_nb"], info["trailing_gemm"])
    assert st["lu_nb"] == info["lu_nb"]
    xo, ro = O.newton(Ns[0], cs[0], "IR16GM", tol=1e-10, lu_nb=info["lu_nb"])
    assert newton_counts_agree(st["newton_iters"], ro) and rel_inf(xs[0], xo) <= 1e-10


def test_batch_full_workload_512_instances():
    """The 512-instance workload (N log-uniform in [64, 2048], c uniform in
    [0.1, 0.999]): every instance converges; at every size the exact discrete
    moment identity (c/2N) sum x = 1 - sqrt(1 - c) holds and the oracle's F
    confirms ||F(x)|| <= 1e-10 ||F(x0)||; the five smallest instances match the
    oracle's Newton to 1e-10."""
    inst = W.batch_instances()
    Ns, cs = [n for n, _ in inst], [c for _, c in inst]
    with nl.Batch(Ns, cs) as B:
        xs, status = B.solve(tol=1e-10)
        info = B.info()
        nb = info["lu_nb"]
        stats = [B.stats(i) for i in range(len(Ns))]
    assert status == nl.NL_OK and info["converged"] == 512
    for N, c, x, st in zip(Ns, cs, xs, stats):
        m = c / (2 * N) * np.sum(x)
        assert abs(m - (1 - math.sqrt(1 - c))) <= 1e-9 / math.sqrt(1 - c)
        f = np.linalg.norm(O.F(N, c, x)) / np.linalg.norm(O.F(N, c, np.ones(N)))
        assert f <= 1e-10 and st["hist"][-1] <= 1e-10
    for k in np.argsort(Ns, kind="stable")[:5]:
        xo, ro = O.newton(Ns[k], cs[k], "IR16GM", tol=1e-10, lu_nb=nb)
        check_instance(stats[k], ro, xs[k], xo)


@pytest.mark.parametrize("mode,omode", [("IR16_GMRES", "IR16GM"), ("FP64LU", "FP64LU")])
def test_batch_instances_leaving_for_the_interchanging_path(mode, omode):
    """lu_path = 1: every instance leaves the batch at its first step (as one
    whose factorisation needs row interchanges does) and is finished on the
    single-instance interchanging path; the results still follow the
    oracle."""
    Ns, cs = small_batch(6, seed=21, n_hi=300)
    with nl.Batch(Ns, cs, lu_nb=64, lu_path=1) as B:
        xs, status = B.solve(tol=1e-10, mode=mode)
        info = B.info()
        stats = [B.stats(i) for i in range(len(Ns))]
    assert status == nl.NL_OK and info["parked_lu"] == len(Ns) and info["parked_ir"] == 0
    for N, c, x, st in zip(Ns, cs, xs, stats):
        xo, ro = O.newton(N, c, omode, tol=1e-10, lu_nb=64)
        check_instance(st, ro, x, xo, lin=(mode != "FP64LU"))
