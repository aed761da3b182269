"""Batched path (grouped LU, grouped triangular solves, graph-captured
Newton over many instances) against the single-instance CUDA path and the
CPU oracle, through the C ABI."""
import json
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


@pytest.mark.parametrize("nb,gemm", [(64, 3), (64, 4), (32, 3), (48, 4), (16, 3)])
def test_lu_grouped_persistent_identical_to_single(nb, gemm):
    """One persistent launch over a device task queue (gemm 3 / 4: 64 x 64 /
    128 x 64 update tiles): factors and pivots bit-for-bit those of the
    single-matrix LU with the SIMT update at the same nb, on the sizes of the
    three-launch test plus one that spans many tiles and several
    off-diagonal quads (N = 1500)."""
    sizes = SIZES + [1500]
    mats = [jacobian16(N, 0.5 + 0.049 * k, 300 + k) for k, N in enumerate(sizes)]
    out, flags = lu_grouped(mats, nb, gemm)
    assert not flags.any()
    for M, (LU, ip) in zip(mats, out):
        N = M.shape[0]
        LUs, ips = lu_single(M, ((N + 63) // 64) * 64, nb, 1)
        assert np.array_equal(ip, np.arange(N)) and np.array_equal(ips, ip)
        assert np.array_equal(LU, LUs), N


@pytest.mark.parametrize("ref_kind", ["single", "grouped"])
def test_lu_grouped_persistent_tcgen05_identical(ref_kind):
    """The persistent launch with 128 x 128 tcgen05 update tiles (gemm 5,
    nb = 64): factors and pivots bit for bit those of the single-matrix LU
    with the tensor-core update at nb = 64, and of the three-launch grouped
    tcgen05 path."""
    sizes = SIZES + [1500, 700]
    mats = [jacobian16(N, 0.5 + 0.049 * k, 700 + k) for k, N in enumerate(sizes)]
    out, flags = lu_grouped(mats, 64, 5)
    assert not flags.any()
    if ref_kind == "grouped":
        ref, rflags = lu_grouped(mats, 64, 2)
        assert not rflags.any()
    for k, (M, (LU, ip)) in enumerate(zip(mats, out)):
        N = M.shape[0]
        LUs, ips = lu_single(M, ((N + 63) // 64) * 64, 64, 2) if ref_kind == "single" else ref[k]
        assert np.array_equal(ip, np.arange(N)) and np.array_equal(ips, ip)
        assert np.array_equal(LU, LUs), N


def test_lu_grouped_persistent_tcgen05_many_matrices_vs_oracle():
    """Many matrices through the tcgen05 persistent launch: the same pivots as
    the oracle's elimination (rounding period 64) and the tensor-core update's
    rule against it: within 8 binary16 roundings (relative to the entry, or to
    2^-11 of the largest pivot), at least 95% of entries identical."""
    g = np.random.default_rng(13)
    Ns = [int(round(math.exp(v))) for v in g.uniform(math.log(20), math.log(900), 40)]
    mats = [jacobian16(N, float(g.uniform(0.1, 0.999)), 900 + k) for k, N in enumerate(Ns)]
    out, flags = lu_grouped(mats, 64, 5)
    assert not flags.any()
    same = total = 0
    for M, (LU, ip) in zip(mats, out):
        LUo, ipo, info, ovf = O.lu16_dev(M, 64)
        assert info == 0 and not ovf and np.array_equal(ip, ipo)
        scale = np.maximum(np.abs(LUo), np.abs(np.diag(LUo)).max() * 2.0 ** -11)
        assert np.max(np.abs(LU - LUo) / scale) <= 8 * 2.0 ** -11
        same += int(np.sum(LU == LUo))
        total += LU.size
    assert same >= 0.95 * total, same / total


def test_lu_grouped_persistent_task_times():
    """nl_debug_grouped_task_times: with timing on, every task of the queue is
    counted once per kind (diagonal blocks, off-diagonal quads, 128 x 128
    tiles) with positive work time; with timing off nothing is counted."""
    Ns = [70, 300, 1000]
    mats = [jacobian16(N, 0.9, 40 + N) for N in Ns]
    nl.grouped_task_times(True)
    lu_grouped(mats, 64, 5)
    t = nl.grouped_task_times(False)
    nd = nq = nt = 0
    for N in Ns:
        for k in range(-(-N // 64)):
            nd += 1
            rest = N - 64 * k - min(64, N - 64 * k)
            if rest > 0:
                nq += 2 * (-(-(-(-rest // 128)) // 4))
                nt += (-(-rest // 128)) ** 2
    assert (t["diag"]["tasks"], t["quad"]["tasks"], t["tile"]["tasks"]) == (nd, nq, nt)
    assert all(t[k]["work_us"] > 0 for k in ("diag", "quad", "tile"))
    lu_grouped(mats, 64, 5)
    t2 = nl.grouped_task_times(False)
    assert all(t2[k]["tasks"] == 0 for k in ("diag", "quad", "tile"))


def test_lu_grouped_persistent_many_matrices_vs_oracle():
    """Many more queue tasks than CTAs (60 matrices, N log-uniform in
    [20, 900]): every matrix equals the oracle's binary16-storage /
    binary32-arithmetic elimination with rounding period nb, exactly."""
    g = np.random.default_rng(11)
    Ns = [int(round(math.exp(v))) for v in g.uniform(math.log(20), math.log(900), 60)]
    mats = [jacobian16(N, float(g.uniform(0.1, 0.999)), 500 + k) for k, N in enumerate(Ns)]
    out, flags = lu_grouped(mats, 32, 4)
    assert not flags.any()
    for M, (LU, ip) in zip(mats, out):
        LUo, ipo, info, ovf = O.lu16_dev(M, 32)
        assert info == 0 and not ovf
        assert np.array_equal(ip, ipo) and np.array_equal(LU, LUo)


def test_lu_grouped_persistent_flags_and_neighbours():
    """In the persistent launch a matrix that needs interchanges is flagged,
    its remaining tasks skip their work but still advance its progress word
    (nothing waits on it), and its neighbours are factored as alone."""
    P, _ = W.pivot_forcing_matrix(150, 3)
    mats = [jacobian16(90, 0.9, 1), O.fl16(P), jacobian16(700, 0.99, 2), O.fl16(W.pivot_forcing_matrix(70, 4)[0])]
    out, flags = lu_grouped(mats, 64, 3)
    assert list(flags) == [0, 1, 0, 1]
    for k in (0, 2):
        N = mats[k].shape[0]
        LUs, ips = lu_single(mats[k], ((N + 63) // 64) * 64, 64, 1)
        assert np.array_equal(out[k][0], LUs) and np.array_equal(out[k][1], ips)


def test_lu_grouped_persistent_rejects_unsupported():
    """The persistent launch takes binary16, nb <= 64 only."""
    A = padded16(jacobian16(100, 0.5, 1), 128)
    ip = torch.empty(100, dtype=torch.int32, device=dev())
    with pytest.raises(RuntimeError):
        nl.lu_grouped([100], [A], [128], [ip], nb=128, gemm=3)


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


def test_batch_autotuner_per_bucket_choice_is_used_and_recorded(tmp_path, monkeypatch):
    """Each N bucket is timed alone for every candidate and takes its fastest;
    every instance's factorisation (stats lu_nb) is its bucket's; the choices
    are written to the tuning table (NL_LU_TUNE_FILE, JSON) and a second
    batch reads them instead of timing, with bit-identical results."""
    Ns, cs = small_batch(10, seed=9)
    path = tmp_path / "tune.json"
    monkeypatch.setenv("NL_LU_TUNE_FILE", str(path))
    with nl.Batch(Ns, cs) as B:
        info0 = B.info()
        xs, status = B.solve(tol=1e-10)
        sts = [B.stats(i) for i in range(len(Ns))]
    assert status == nl.NL_OK
    bks = info0["buckets"]
    assert len(bks) >= 2 and sum(b["count"] for b in bks) == len(Ns)
    for k, b in enumerate(bks):
        cands = [t for t in info0["tune"] if t[3] == k]
        assert len(cands) >= 2 and not b["cached"]
        best = min(cands, key=lambda t: t[2])
        assert (best[0], best[1]) == (b["nb"], b["gemm"])
    bounds = [b["nmax"] for b in bks]
    for i, N in enumerate(Ns):
        k = next(j for j, m in enumerate(bounds) if N <= m)
        assert sts[i]["lu_nb"] == bks[k]["nb"]
    assert (info0["lu_nb"], info0["trailing_gemm"]) == (bks[-1]["nb"], bks[-1]["gemm"])
    xo, ro = O.newton(Ns[0], cs[0], "IR16GM", tol=1e-10, lu_nb=sts[0]["lu_nb"])
    assert newton_counts_agree(sts[0]["newton_iters"], ro) and rel_inf(xs[0], xo) <= 1e-10
    table = json.loads(path.read_text())["entries"]
    assert len(table) == len(bks)
    with nl.Batch(Ns, cs) as B2:
        info1 = B2.info()
        xs2, _ = B2.solve(tol=1e-10)
    assert info1["tune_count"] == 0 and all(b["cached"] for b in info1["buckets"])
    assert [(b["nb"], b["gemm"]) for b in info1["buckets"]] == [(b["nb"], b["gemm"]) for b in bks]
    for a, b in zip(xs, xs2):
        assert np.array_equal(a, b)


def test_batch_tuning_table_unreadable_is_ignored(tmp_path, monkeypatch):
    """A tuning table that is not ours (or holds choices this device cannot
    run) is ignored: the batch times its buckets and overwrites it."""
    path = tmp_path / "tune.json"
    path.write_text('{"entries": {"x": {"nb": 999, "gemm": 7, "ms": 1.0}}}\nnot json at all\n')
    monkeypatch.setenv("NL_LU_TUNE_FILE", str(path))
    Ns, cs = small_batch(4, seed=2)
    with nl.Batch(Ns, cs) as B:
        info = B.info()
        _, status = B.solve(tol=1e-10)
    assert status == nl.NL_OK and info["tune_count"] >= 2 and not any(b["cached"] for b in info["buckets"])
    assert len(json.loads(path.read_text())["entries"]) >= 1


@pytest.mark.parametrize("gemm,ref", [(3, 1), (4, 1), (5, 2)])
def test_batch_persistent_grouped_lu_in_graph_equals_three_launch(gemm, ref):
    """The persistent grouped-LU launch inside the batch graph (conditional
    WHILE body, buckets side by side): every instance's iterate bit for bit
    that of the three-launch grouped LU with the same update arithmetic
    (SIMT for 3 / 4, tcgen05 for 5) at the same nb."""
    Ns, cs = small_batch(12, seed=21)
    with nl.Batch(Ns, cs, lu_nb=64, trailing_gemm=ref) as B1:
        x1, s1 = B1.solve(tol=1e-10)
    with nl.Batch(Ns, cs, lu_nb=64, trailing_gemm=gemm) as B2:
        x2, s2 = B2.solve(tol=1e-10)
        info = B2.info()
    assert s1 == s2 == nl.NL_OK and all(b["gemm"] == gemm for b in info["buckets"])
    for a, b in zip(x1, x2):
        assert np.array_equal(a, b)


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
