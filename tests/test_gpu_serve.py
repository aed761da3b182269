"""Serving loop (nl_server_*): admission by device-memory footprint,
concurrent requests on their own streams, results independent of the mix,
parity with the oracle, latency accounting."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16051_gb300 import nl
from tests.conftest import newton_counts_agree
from paper_2307_16051_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()


def rel_inf(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


PROBES = [(256, 0.9), (1024, 0.9999), (256, 0.5), (512, 0.99)]


def solve_alone(N, c):
    with nl.Server(max_inflight=1) as S:
        rid = S.submit(N, c)
        S.start()
        x, st, info = S.result(rid)
    assert info["status"] == nl.NL_OK
    return x, st


def test_result_same_alone_and_in_the_mix():
    """Each probe request gives the same iterate alone and when it shares the
    GPU with a stream of other requests (concurrent slots, handle reuse and
    eviction under a tight memory budget): bitwise equal, hence within the
    1e-10 parity tolerance."""
    alone = {p: solve_alone(*p) for p in PROBES}
    budget = 3 * nl.footprint_bytes(1024) + 2 * nl.footprint_bytes(512)
    mix = [(256, 0.7), (1024, 0.95), (512, 0.6), (256, 0.999), (1024, 0.5), (512, 0.9)] * 3
    with nl.Server(budget_bytes=budget, max_inflight=4) as S:
        ids = [S.submit(N, c, arrival_s=0.002 * k) for k, (N, c) in enumerate(mix)]
        pid = {p: S.submit(p[0], p[1], arrival_s=0.005 * (k + 1)) for k, p in enumerate(PROBES)}
        S.start()
        assert S.drain(120.0) == nl.NL_OK
        info = S.info()
        for p, rid in pid.items():
            x, st, ri = S.result(rid)
            xa, sa = alone[p]
            assert ri["status"] == nl.NL_OK and st["newton_iters"] == sa["newton_iters"]
            assert np.array_equal(x, xa) and rel_inf(x, xa) <= 1e-10
        for rid in ids:
            assert S.result(rid)[2]["status"] == nl.NL_OK
    assert info["completed"] == len(mix) + len(PROBES) and info["failed"] == 0
    assert info["bytes_peak"] <= budget and info["inflight_peak"] >= 2
    assert info["handles_created"] < info["completed"]


def test_served_results_match_oracle():
    reqs = [(256, 0.5), (300, 0.99), (200, 0.9999), (128, 0.999)]
    with nl.Server(max_inflight=4) as S:
        ids = [S.submit(N, c) for N, c in reqs]
        S.start()
        for (N, c), rid in zip(reqs, ids):
            x, st, ri = S.result(rid)
            xo, ro = O.newton(N, c, "IR16GM", tol=1e-10)
            assert ri["status"] == nl.NL_OK and ro["status"] == 0
            assert newton_counts_agree(st["newton_iters"], ro)
            for a, b in zip(st["lin_iters"], ro["lin_iters"]):
                assert abs(a - b) <= 1
            assert rel_inf(x, xo) <= 1e-10


def test_admission_respects_the_memory_budget():
    """A budget that holds two N = 1024 handles: never more than two such
    requests on the device, never more bytes than the budget; a request
    larger than the budget is refused at submission."""
    fp = nl.footprint_bytes(1024)
    with nl.Server(budget_bytes=2 * fp + fp // 2, max_inflight=6) as S:
        ids = [S.submit(1024, 0.9) for _ in range(8)]
        with pytest.raises(nl.NLError):
            S.submit(4096, 0.9)
        S.start()
        assert S.drain(120.0) == nl.NL_OK
        info = S.info()
        spans = sorted((S.result(r)[2]["t_admit_s"], S.result(r)[2]["t_done_s"]) for r in ids)
    assert info["inflight_peak"] <= 2 and info["bytes_peak"] <= 2 * fp + fp // 2
    assert info["handles_created"] == 2
    for k, (a, _) in enumerate(spans):
        live = sum(1 for (a2, d2) in spans if a2 <= a < d2)
        assert live <= 2


def test_short_poisson_trace_latency_accounting():
    """A short Poisson trace of the serving workload's shape (two smallest
    sizes): every request completes, latency = completion - arrival >= the
    request's own device time, and the percentiles are ordered."""
    trace = W.serving_trace(seed=7, rate_per_s=150.0, duration_s=1.0, sizes=(256, 1024), probs=(0.6, 0.4))
    with nl.Server(max_inflight=8) as S:
        ids = [S.submit(N, c, arrival_s=t) for t, N, c in trace]
        S.start()
        assert S.drain(120.0) == nl.NL_OK
        info = S.info()
        for rid in ids:
            x, st, ri = S.result(rid)
            assert ri["status"] == nl.NL_OK
            assert ri["t_admit_s"] >= ri["t_arrive_s"] - 1e-6 and ri["t_done_s"] >= ri["t_admit_s"]
            assert ri["latency_ms"] >= st["t_total_ms"] * 0.999
    assert info["completed"] == len(trace)
    assert 0 < info["p50_ms"] <= info["p99_ms"] and info["solves_per_s"] > 0


def test_serving_trace_slice_full_sizes():
    """The first 0.5 s of the serving workload itself (all four sizes, up to
    N = 16384, replayed through the bench's server configuration): every
    request converges; each result meets ||F(x)|| <= 1e-10 ||F(x0)|| under the
    oracle's double-precision F and the exact moment identity; the small ones
    match the oracle's Newton to 1e-10."""
    import math
    trace = W.serving_trace(duration_s=0.5)
    assert {N for _, N, _ in trace} >= {256, 1024, 4096}
    with nl.Server(budget_bytes=96 << 30, max_inflight=8) as S:
        ids = [S.submit(N, c, arrival_s=t) for t, N, c in trace]
        S.start()
        assert S.drain(300.0) == nl.NL_OK
        results = [S.result(r) for r in ids]
    checked_oracle = 0
    for (t, N, c), (x, st, ri) in zip(trace, results):
        assert ri["status"] == nl.NL_OK
        m = c / (2 * N) * np.sum(x)
        assert abs(m - (1 - math.sqrt(1 - c))) <= 1e-9 / math.sqrt(1 - c)
        f = np.linalg.norm(O.F(N, c, x)) / np.linalg.norm(O.F(N, c, np.ones(N)))
        assert f <= 1e-10
        if N == 256 and checked_oracle < 4:
            xo, ro = O.newton(N, c, "IR16GM", tol=1e-10)
            assert newton_counts_agree(st["newton_iters"], ro) and rel_inf(x, xo) <= 1e-10
            checked_oracle += 1
