"""Benchmark: three-precision Newton solves on GB300 versus FP64-LU Newton.

Workload (one "step"): the paper's conditioning sweep of the H-equation
(Section 3, eq. (3.2)) at N = 4096, c in {.5, .9, .99, .9999, .999999},
x0 = ones, each solved to ||F||/||F0|| <= 1e-10 with GMRES-IR16 (restart 30,
inner tolerance 1e-4, eta = 1e-4): five Newton solves per step.

value     : solves/s with x0/x in HBM (nl_solve_device), CUDA events.
e2e       : solves/s through nl_solve with host buffers (copies included).
per_c     : per c, the counts, and each result's error against the oracle's
            FP64-LU solution (tests/golden/sweep_n4096_x.npy, oracle-written).
baselines : the same sweep with FP64-LU Newton and with IR16 on the same GPU,
            and the CPU oracle on the host cores (the whole sweep, measured).
ablations : the section 2.3 variants and the scaling into the binary16 range.
batched   : the 512-instance batch (one graph-captured batched solve), and
            the same batch with FP64-LU Newton.
serving   : the serving trace's first --serve-seconds seconds replayed in
            real time through the request loop: p50/p99 latency, solves/s;
            FP64-LU Newton served over the same window.
large     : GMRES-IR16 at N = 32768, c = .99, autotuned panel width (median of
            three solves; LU TFLOP/s, residual / triangular-solve GB/s), the
            scaled variant, and FP64-LU Newton on the same GPU.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# Hardware work queues for the concurrent solves (read when the CUDA context is
# created): each solve has its stream and its LU look-ahead's side stream, and
# with CUDA's default of 8 queues the sweep's ten streams (the server's up to
# sixteen) would share queues and wait on one another's unrelated launches.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

SWEEP = (0.5, 0.9, 0.99, 0.9999, 0.999999)
N_BENCH = 4096
TOL = 1e-10
WORKLOAD = ("H-equation (eq. 3.2) N=4096, c in {.5,.9,.99,.9999,.999999}, x0=ones, "
            "to ||F||/||F0||<=1e-10, GMRES-IR16 restart 30 inner tol 1e-4, eta 1e-4")
METRIC = "Newton solves/s to ||F||/||F0||<=1e-10 (N=4096 conditioning sweep, three-precision GMRES-IR16)"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a while to start: wait for its first line (taken before the timed
            # region, so dropped), then every later sample falls inside the region
            t0 = time.time()
            while not self.lines and time.time() - t0 < 10.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines = []
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x 2 flop/FMA x max SM clock


def kernel_rooflines(nl, step, N, hbm_peak, tc_peak, lookahead=True):
    """Time each kernel class of one GMRES-IR16 sweep with CUDA events (the
    library brackets every launch of the class on its stream) and set the
    algorithmic work of one launch against its roofline.  With the LU's
    look-ahead each trailing update is two launches: the cross (the first
    128-row and 128-column tile strips, class k_tc_gemm_x) and the rest
    (k_tc_gemm)."""
    NB, T2 = 128, 128
    out = {}
    # algorithmic work per launch at N = 4096, nb = 128 (averaged over the 32 panels)
    panels = [(K, min(NB, N - K)) for K in range(0, N, NB)]
    diag_flop = sum(2.0 * w ** 3 / 3.0 for _, w in panels) / len(panels)
    off = [(N - K - w, w) for K, w in panels if N - K - w > 0]
    off_flop = sum(2.0 * 2 * r * w * w / 2.0 for r, w in off) / len(off)          # L21 and U12 solves
    gemm_flop = sum(2.0 * r * r * w for r, w in off) / len(off)
    rest = [(r, w) for r, w in off if r > T2]
    rest_flop = sum(2.0 * (r - T2) ** 2 * w for r, w in rest) / max(1, len(rest))
    cross_flop = sum(2.0 * (r * r - max(r - T2, 0) ** 2) * w for r, w in off) / len(off)
    nblk = (N + T2 - 1) // T2
    trsv_bytes = (N * N / 2.0) * 2 + nblk * T2 * T2 * 4 + 3 * N * 4                 # fp16 triangle + diag inverses + vectors
    gemv_bytes = 4.0 * N * N + 3 * 4.0 * N                                          # fp32 J and vectors
    spec = {
        "k_diag_lu16": ("alu", diag_flop, FP32_PEAK_TFLOPS, "TFLOP/s", "derived fp32 FMA peak (152 SMs x 128 lanes x 2 x 2.07 GHz)"),
        "k_offdiag16": ("alu", off_flop, FP32_PEAK_TFLOPS, "TFLOP/s", "derived fp32 FMA peak"),
        "k_panel16": ("alu", diag_flop + off_flop, FP32_PEAK_TFLOPS, "TFLOP/s",
                      "derived fp32 FMA peak (diagonal block and off-diagonal solves in one launch)"),
        "k_tc_gemm": ("tensor", rest_flop if lookahead else gemm_flop, tc_peak, "TFLOP/s",
                      "measured bf16 dense (fp16 same rate)"),
        "k_tc_gemm_x": ("tensor", cross_flop, tc_peak, "TFLOP/s", "measured bf16 dense (fp16 same rate)"),
        "k_trsv_cl": ("hbm", trsv_bytes, hbm_peak, "GB/s", "measured copy bandwidth"),
        "k_trsv_mb": ("hbm", trsv_bytes, hbm_peak, "GB/s", "measured copy bandwidth"),
        "k_gemv_residual": ("hbm", gemv_bytes, hbm_peak, "GB/s", "measured copy bandwidth"),
    }
    for name, (bound, work, peak, unit, kind) in spec.items():
        nl.kernel_timing(name)
        step("GMRESIR16")
        n, ms = nl.kernel_timing(None)
        if n == 0:
            continue
        avg_s = ms / n / 1e3
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        ach = work / avg_s / scale
        out[name] = {"kernel": name, "bound": bound, "launches": n, "total_ms": ms, "avg_us": avg_s * 1e6,
                     "work_per_launch": work, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                     "traffic": None, "peak_kind": kind}
    return out


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None."""
    try:
        for line in open(os.path.join(ROOT, "profiles", "ncu_traffic_per_launch.txt")):
            p = line.split()
            if len(p) == 2 and not line.startswith("#") and p[0] == kernel:
                return int(p[1])
    except OSError:
        pass
    return None


GROUPED_KIND = {1: "simt, 3 launches per outer step", 2: "tcgen05, 3 launches per outer step",
                3: "one persistent launch, 64x64 simt tiles", 4: "one persistent launch, 128x64 simt tiles",
                5: "one persistent launch, 128x128 tcgen05 tiles"}


def bench_batched(nl, W, torch, dev, steps, warmup, tc_peak, fp64=True):
    """The 512-instance batch (N log-uniform in [64, 2048], c uniform in
    [0.1, 0.999], x0 = ones, seed 230716051): one graph-captured batched solve
    per step, x in HBM; the same batch with FP64-LU Newton on the same GPU."""
    inst = W.batch_instances()
    Ns, cs = [n for n, _ in inst], [c for _, c in inst]
    B = nl.Batch(Ns, cs)
    tot = int(sum(Ns))
    xout = torch.empty(tot, device=dev, dtype=torch.float64)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev, dtype=torch.float32)
    for _ in range(max(1, warmup)):
        B.solve_device(xout, tol=TOL, mode="IR16_GMRES")
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = B.solve_device(xout, tol=TOL, mode="IR16_GMRES")
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    info = B.info()
    lu_flop = sum(2.0 * n ** 3 / 3.0 for n in Ns)
    out = {"workload": "512 instances, N log-uniform [64, 2048] (seed 230716051), c uniform [0.1, 0.999], x0=ones, "
                       "IR16 with GMRES-IR16 fallback, eta 1e-4, to 1e-10",
           "status": nl.STATUS_NAMES[st], "solves_per_s": len(Ns) / (statistics.median(ms) / 1e3),
           "ms_per_batch": statistics.median(ms), "converged": info["converged"],
           "parked_lu": info["parked_lu"], "parked_ir": info["parked_ir"], "newton_rounds": info["newton_rounds"],
           "ir_rounds": info["ir_rounds"], "gpu_launches": info["gpu_launches"],
           "graph": "one CUDA graph per solve: WHILE(Newton) { J, grouped LU, WHILE(IR) {...}, update }",
           "autotune": [{"bucket_nmax": info["buckets"][t[3]]["nmax"], "nb": t[0], "gemm": GROUPED_KIND[t[1]],
                         "bucket_lu_ms": t[2]} for t in info["tune"]],
           "buckets": [{"nmax": b["nmax"], "count": b["count"], "nb": b["nb"], "gemm": GROUPED_KIND[b["gemm"]],
                        "from_table": bool(b["cached"])} for b in info["buckets"]],
           "lu_nb": info["lu_nb"], "trailing_gemm": GROUPED_KIND[info["trailing_gemm"]]}
    if info["lu16_ms"] > 0:
        tf = lu_flop / (info["lu16_ms"] / 1e3) / 1e12
        out["grouped_lu"] = {"ms": info["lu16_ms"], "achieved": tf, "peak": tc_peak, "unit": "TFLOP/s",
                             "frac": tf / tc_peak,
                             "work": "sum of 2N^3/3 over the 512 Jacobians at x0; every N bucket's grouped LU "
                                     "side by side on its own stream, CUDA events around the whole"}
    if fp64:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st64 = B.solve_device(xout, tol=TOL, mode="FP64LU")
        e1.record()
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        i64 = B.info()
        out["fp64lu"] = {"status": nl.STATUS_NAMES[st64], "solves_per_s": len(Ns) / (ms64 / 1e3), "ms_per_batch": ms64,
                         "newton_rounds": i64["newton_rounds"]}
        out["speedup_vs_fp64lu"] = ms64 / out["ms_per_batch"]
    B.close()
    return out


def bench_large(nl, torch, dev, hbm_peak, tc_peak, N=32768, c=0.99, fp64=True, reps=3):
    """GMRES-IR16 solves at N = 32768, c = .99 with the autotuned panel
    width: time to 1e-10 (the median of `reps` solves after a warm-up), the
    factorisation's TFLOP/s, and the residual GEMV and triangular solves'
    GB/s (CUDA events on every launch); the same solve with the scaling into
    the binary16 range; and FP64-LU Newton on the same GPU (one solve)."""
    s = nl.Solver(N, c, lu_nb=-1)
    x = torch.empty(N, device=dev, dtype=torch.float64)
    s.solve_device(x, tol=TOL, mode="GMRESIR16")  # warm-up
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        status = s.solve_device(x, tol=TOL, mode="GMRESIR16")
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    st = s.stats()
    lu_flop = 2.0 * N ** 3 / 3.0
    lu_ms = st["t_lu_ms"] / max(1, st["newton_iters"])
    lu_tf = lu_flop / (lu_ms / 1e3) / 1e12
    kern = {}
    T2 = 128
    nblk = (N + T2 - 1) // T2
    work = {"k_gemv_residual": 4.0 * N * N + 12.0 * N,
            "k_trsv_cl": (N * N / 2.0) * 2 + nblk * T2 * T2 * 4 + 12.0 * N,
            "k_trsv_mb": (N * N / 2.0) * 2 + nblk * T2 * T2 * 4 + 12.0 * N,
            "k_tc_gemm": None}
    for name in ("k_gemv_residual", "k_trsv_cl", "k_trsv_mb", "k_tc_gemm"):
        nl.kernel_timing(name)
        s.solve_device(x, tol=TOL, mode="GMRESIR16")
        n, kms = nl.kernel_timing(None)
        if n:
            k = {"launches": n, "total_ms": kms, "avg_us": kms / n * 1e3}
            if work[name]:
                gbs = work[name] / (kms / n / 1e3) / 1e9
                k.update({"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                          "work_per_launch": work[name]})
            kern[name] = k
    out = {"workload": f"H-equation N={N}, c={c}, x0=ones, GMRES-IR16 (restart 30, tol 1e-4), eta 1e-4, to 1e-10, "
                       "panel width autotuned", "status": nl.STATUS_NAMES[status], "ms_to_solution": ms,
           "ms_solves": times, "timing": f"median of {reps} solves after one warm-up solve",
           "newton": st["newton_iters"], "lin_iters": st["lin_iters"], "lu_nb": st["lu_nb"],
           "autotune": [{"nb": nb, "lu_ms": t} for nb, t in st["lu_tune"]],
           "lu": {"ms_per_factorisation": lu_ms, "achieved": lu_tf, "peak": tc_peak, "unit": "TFLOP/s",
                  "frac": lu_tf / tc_peak, "work": "2N^3/3"},
           "t_f_ms": st["t_f_ms"], "t_jac_ms": st["t_jac_ms"], "t_lu_ms": st["t_lu_ms"], "t_lin_ms": st["t_lin_ms"],
           "kernels": kern, "final_rel_res": st["hist"][-1]}
    xg = x.cpu().numpy()
    s.close()
    # the scaled factorisation (scale_fp16 = 1): one warm-up, one timed solve
    with nl.Solver(N, c, lu_nb=-1, scale_fp16=1) as ss:
        ss.solve_device(x, tol=TOL, mode="GMRESIR16")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sst = ss.solve_device(x, tol=TOL, mode="GMRESIR16")
        e1.record()
        torch.cuda.synchronize()
        S2 = ss.stats()
        out["scaled"] = {"status": nl.STATUS_NAMES[sst], "ms_to_solution": e0.elapsed_time(e1),
                         "newton": S2["newton_iters"], "lin_iters": S2["lin_iters"], "final_rel_res": S2["hist"][-1],
                         "max_rel_diff_vs_unscaled": float(abs(x.cpu().numpy() - xg).max() / abs(xg).max()),
                         "note": "J_h = fl16(R J32) with power-of-two row factors; at this N nearly every "
                                 "off-diagonal entry of the unscaled J_h is a binary16 subnormal"}
    if fp64:
        s64 = nl.Solver(N, c)
        torch.cuda.synchronize()
        e0.record()
        st64 = s64.solve_device(x, tol=TOL, mode="FP64LU")
        e1.record()
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        x64 = x.cpu().numpy()
        out["fp64lu"] = {"status": nl.STATUS_NAMES[st64], "ms_to_solution": ms64, "newton": s64.stats()["newton_iters"],
                         "lu_ms_per_factorisation": s64.stats()["t_lu_ms"] / max(1, s64.stats()["newton_iters"]),
                         "timing": "one solve (no warm-up: the FP64 LU dominates, about 18 s per factorisation)"}
        out["speedup_vs_fp64lu"] = ms64 / ms
        out["err_vs_gpu_fp64lu"] = float(abs(xg - x64).max() / abs(x64).max())
        s64.close()
    return out


def bench_serving(nl, W, seconds, mode="IR16_GMRES", drain_s=120.0, max_inflight=8):
    """The serving trace (Poisson 200 req/s, N from {256, 1024, 4096, 16384}
    with p = {.5, .3, .15, .05}, c uniform [.5, .9999], seed 16051), cut to
    its first `seconds` seconds and replayed in real time."""
    trace = W.serving_trace(duration_s=seconds)
    with nl.Server(budget_bytes=96 << 30, max_inflight=max_inflight, mode=mode) as S:
        ids = [S.submit(N, c, arrival_s=t) for t, N, c in trace]
        S.start()
        rc = S.drain(seconds + drain_s)  # the arrivals span `seconds`; then at most drain_s more
        info = S.info()
        per_n = {}
        for rid, (t, N, c) in zip(ids, trace):
            x, st, ri = S.result(rid, wait=False)
            if ri["status"] == nl.NL_OK:
                per_n.setdefault(N, []).append(ri["latency_ms"])
    import numpy as np
    out = {"workload": f"Poisson 200 req/s, first {seconds:g} s of the 60 s trace (seed 16051), N from "
                       "{256,1024,4096,16384} p={.5,.3,.15,.05}, c uniform [.5,.9999], to 1e-10",
           "mode": mode, "requests": len(trace), "completed": info["completed"], "failed": info["failed"],
           "drained": rc == nl.NL_OK, "p50_ms": info["p50_ms"], "p99_ms": info["p99_ms"], "mean_ms": info["mean_ms"],
           "solves_per_s": info["solves_per_s"], "span_s": info["span_s"], "inflight_peak": info["inflight_peak"],
           "bytes_peak": info["bytes_peak"], "handles_created": info["handles_created"],
           "per_N": {str(n): {"count": len(v), "p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99))}
                     for n, v in sorted(per_n.items())},
           "admission": f"device-memory footprint (budget 96 GiB), {max_inflight} slots, smallest N first with a "
                        "250 ms starvation bound, high-priority streams for N <= 1024"}
    return out


def golden_x():
    """The oracle's FP64-LU solutions of the sweep (written by
    tests/golden/make_golden.py from the CPU oracle alone), or None."""
    import numpy as np
    p = os.path.join(ROOT, "tests", "golden", "sweep_n4096_x.npy")
    try:
        return np.load(p)
    except OSError:
        return None


def golden_counts():
    p = os.path.join(ROOT, "tests", "golden", "sweep_n4096.json")
    try:
        g = json.load(open(p))
        return {k: (v["newton_iters"], v["hist"]) for k, v in g["cases"].items()}
    except (OSError, ValueError, KeyError):
        return None


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("NL_BENCH_GLOO") != "1" else "gloo")
    return ws, rank, local


def barrier_max(value, ws):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample():
    """The oracle as it stands on the host cores, timed on the workload
    itself: the five GMRES-IR16 Newton solves of the sweep (N = 4096, c in
    SWEEP, x0 = ones, to 1e-10), one after another, each complete."""
    from oracle import oracle as O
    O.build()
    t = time.time()
    steps = 0
    for c in SWEEP:
        _, r = O.newton(N_BENCH, c, "GMRESIR16", tol=TOL)
        steps += r["newton_iters"]
    dt = time.time() - t
    return {"value": len(SWEEP) / dt, "unit": "solves/s", "cores": O.num_threads(), "kind": "oracle",
            "seconds": dt,
            "sample": (f"the whole sweep measured: 5 complete oracle GMRES-IR16 Newton solves at N=4096 (c in "
                       f"{list(SWEEP)}, {steps} Newton steps in all; J, binary16-storage/binary32-arithmetic LU, "
                       f"GMRES-IR) in {dt:.1f} s on {O.num_threads()} threads")}


def run_reference(args, ws, rank):
    """The oracle arm: each step is one complete oracle GMRES-IR16 Newton
    solve of the sweep at N = 4096 (the steps go through the five c in turn,
    so K = 5m steps are m whole sweeps), timed on the host cores; the warm-up
    steps solve at the same size.  value = solves / measured seconds."""
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    for k in range(args.warmup):
        O.newton(N_BENCH, SWEEP[k % len(SWEEP)], "GMRESIR16", tol=TOL)
    times = []
    for k in range(args.steps):
        t = time.time()
        O.newton(N_BENCH, SWEEP[k % len(SWEEP)], "GMRESIR16", tol=TOL)
        times.append(time.time() - t)
    total = sum(times)
    value = len(times) / total
    sample = (f"{len(times)} complete oracle GMRES-IR16 Newton solves at N=4096, c cycling through {list(SWEEP)}, "
              f"measured: {total:.1f} s in all on {O.num_threads()} threads (no extrapolation)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16/f32/f64 (emulated)",
            "data": "synthetic", "config": {"workload": WORKLOAD, "N": N_BENCH, "c": list(SWEEP),
                                            "step": "one complete solve (c cycling through the sweep)"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--lu-nb", type=int, default=0, help="LU outer block (0: library default)")
    ap.add_argument("--lu-stream", type=int, default=0,
                    help="panel launch: 0 library default, 256 streaming CTAs of 256 rows, -1 two launches")
    ap.add_argument("--lu-lookahead", type=int, default=0,
                    help="LU look-ahead: 0 library default (on), -1 one trailing update per panel")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-instance batched workload")
    ap.add_argument("--no-large", action="store_true", help="skip the N=32768 single solve")
    ap.add_argument("--no-large-fp64", action="store_true", help="skip FP64-LU Newton at N=32768 (about 2 minutes)")
    ap.add_argument("--serve-seconds", type=float, default=30.0,
                    help="seconds of the serving trace to replay (0: skip serving)")
    ap.add_argument("--serve-fp64-seconds", type=float, default=30.0,
                    help="seconds of the serving trace to replay with FP64-LU Newton (0: skip)")
    args = ap.parse_args()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import numpy as np
    import torch

    from paper_2307_16051_gb300 import nl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbm_peak, tc_peak, tc_sust, peak_kind = peaks()
    # the five solves of a step are independent problems: each runs on its own
    # stream, driven by its own host thread, so that their latency-bound
    # factorisations share the GPU (per-solve times are reported separately).
    # Larger c takes more Newton steps, so the step's time is that solve's
    # latency: its stream gets the highest priority (lower number = higher).
    order = sorted(SWEEP)
    streams = {c: torch.cuda.Stream(device=dev, priority=-order.index(c)) for c in SWEEP}
    solvers = {c: nl.Solver(N_BENCH, c, stream=streams[c], lu_nb=args.lu_nb, lu_stream=args.lu_stream,
                            lu_lookahead=args.lu_lookahead) for c in SWEEP}
    xdev = {c: torch.empty(N_BENCH, device=dev, dtype=torch.float64) for c in SWEEP}
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev, dtype=torch.float32)
    import concurrent.futures as cf
    pool = cf.ThreadPoolExecutor(max_workers=len(SWEEP))

    # end-to-end inputs and outputs in pinned host memory: x0 = ones is copied in and x copied out
    x0_host = {c: torch.ones(N_BENCH, dtype=torch.float64).pin_memory().numpy() for c in SWEEP}
    x_host = {c: torch.empty(N_BENCH, dtype=torch.float64).pin_memory().numpy() for c in SWEEP}

    def one(c, mode, device_api):
        if device_api:
            solvers[c].solve_device(xdev[c], tol=TOL, mode=mode)
        else:
            solvers[c].solve(tol=TOL, mode=mode, x0=x0_host[c], out=x_host[c])
        return solvers[c].stats()

    def step(mode, device_api=True, concurrent=True):
        if not concurrent:
            return {c: one(c, mode, device_api) for c in SWEEP}
        futs = {c: pool.submit(one, c, mode, device_api) for c in SWEEP}
        return {c: f.result() for c, f in futs.items()}

    def timed(mode, k, device_api=True, concurrent=True):
        ms = []
        stats = None
        for _ in range(k):
            flush.fill_(1.0)  # L2 flush between steps (256 MiB write)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            stats = step(mode, device_api, concurrent)
            e1.record()  # after every solve returned (each synchronises its stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, stats

    for _ in range(max(3, args.warmup)):
        step("GMRESIR16")
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    with ClockSampler(local) as clk:
        ms, stats = timed("GMRESIR16", args.steps)
    torch.cuda.synchronize()
    ms_step = barrier_max(sum(ms) / len(ms), ws)
    solves = len(SWEEP) * ws
    value = solves / (ms_step / 1e3)
    # end to end through the host-buffer API
    ms_e2e, _ = timed("GMRESIR16", max(1, args.steps), device_api=False)
    ms_e2e_step = barrier_max(sum(ms_e2e) / len(ms_e2e), ws)
    e2e = {"value": solves / (ms_e2e_step / 1e3), "unit": "solves/s", "h2d_bytes_per_step": len(SWEEP) * N_BENCH * 8,
           "d2h_bytes_per_step": len(SWEEP) * N_BENCH * 8,
           "path": "nl_solve with x0 and x in pinned host memory (copies inside the timed region)"}
    # per-phase device times of the GMRES-IR16 sweep
    lu_ms = sum(s["t_lu_ms"] for s in stats.values())
    n_lu = sum(s["newton_iters"] for s in stats.values())
    launches = sum(s["gpu_launches"] for s in stats.values())
    # sequential solves for the per-launch kernel timing (event pairs per kernel class)
    kern = kernel_rooflines(nl, lambda mode: step(mode, True, False), N_BENCH, hbm_peak, tc_peak,
                            lookahead=args.lu_lookahead == 0)
    ms_seq, _ = timed("GMRESIR16", 1, concurrent=False)
    dom = max(kern.values(), key=lambda k: k["total_ms"])
    roofline = {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    roofline["traffic"] = ncu_traffic(dom["kernel"]) if dom["kernel"] in ("k_diag_lu16", "k_offdiag16", "k_panel16") else None
    roofline.update({"kernel": dom["kernel"], "launches": dom["launches"], "avg_us": dom["avg_us"],
                     "work_per_launch": dom["work_per_launch"], "peak_kind": dom["peak_kind"]})
    lu_flops = 2.0 * N_BENCH ** 3 / 3.0
    lu_tf = lu_flops / (lu_ms / n_lu / 1e3) / 1e12 if n_lu else 0.0
    roofline_lu = {"bound": "tensor", "achieved": lu_tf, "peak": tc_peak, "unit": "TFLOP/s", "frac": lu_tf / tc_peak,
                   "note": "whole binary16 LU (2N^3/3 flop) over its device time per factorisation"}
    X64 = golden_x()
    GC = golden_counts()

    def errors(mode, st_by_c):
        """Per c: ||x - x_oracle64||_inf / ||x_oracle64||_inf of the results now in xdev, and
        how the Newton count compares with the oracle's for the same mode."""
        out = {}
        for k, c in enumerate(SWEEP):
            e = {}
            if X64 is not None:
                x = xdev[c].cpu().numpy()
                err = float(np.max(np.abs(x - X64[k])) / np.max(np.abs(X64[k])))
                e["err_vs_fp64_oracle"] = err if math.isfinite(err) else None  # (a diverged comparison column)
            if mode and GC is not None and f"{c}/{mode}" in GC:
                n_or, h_or = GC[f"{c}/{mode}"]
                n = st_by_c[c]["newton_iters"]
                e["newton_oracle"] = n_or
                e["newton_match"] = ("equal" if n == n_or else
                                     ("one apart: oracle residual at the smaller count within 2x of tol"
                                      if abs(n - n_or) == 1 and h_or[min(n, n_or)] <= 2 * TOL else "DIFFERENT"))
            out[str(c)] = e
        return out

    err_gm = errors("GMRESIR16", stats)
    per_c = {str(c): {"newton": s["newton_iters"], "lin_iters": s["lin_iters"], "ms": s["t_total_ms"],
                      "final_rel_res": s["hist"][-1], "lu_ms": s["t_lu_ms"], "lin_ms": s["t_lin_ms"],
                      **err_gm[str(c)]}
             for c, s in stats.items()}
    extra = {}
    if not args.no_fp64:
        ms64, st64 = timed("FP64LU", 1)
        extra["fp64lu"] = {"solves_per_s": len(SWEEP) / (sum(ms64) / 1e3), "ms_per_sweep": sum(ms64),
                           "per_c_ms": {str(c): s["t_total_ms"] for c, s in st64.items()},
                           "newton": {str(c): s["newton_iters"] for c, s in st64.items()},
                           "vs_oracle": errors("FP64LU", st64)}
        extra["speedup_vs_fp64lu"] = extra["fp64lu"]["ms_per_sweep"] / ms_step
    msir, stir = timed("IR16", 1)
    err_ir = errors("IR16", stir)
    extra["ir16"] = {"ms_per_sweep": sum(msir), "per_c": {str(c): {"status": nl.STATUS_NAMES[s["status"]],
                                                                     "newton": s["newton_iters"], "ms": s["t_total_ms"],
                                                                     "lin_iters": s["lin_iters"], "lin_ms": s["t_lin_ms"],
                                                                     **err_ir[str(c)]}
                                                            for c, s in stir.items()}}
    # the paper's two-precision comparison columns (Section 1.3): one solve per step in the
    # factorisation's precision, no refinement
    def one_tp(c, mode):
        try:
            solvers[c].solve_device(xdev[c], tol=TOL, mode=mode)
        except nl.NLError:
            pass  # a non-finite residual or a zero pivot: the status is in the stats
        return solvers[c].stats()

    extra["two_precision"] = {}
    for mode in ("F32", "F16"):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        futs = {c: pool.submit(one_tp, c, mode) for c in SWEEP}
        stm = {c: f.result() for c, f in futs.items()}
        e1.record()
        torch.cuda.synchronize()
        err_tp = errors(None, stm)  # the error against the FP64 oracle is stated for every column
        extra["two_precision"][mode] = {
            "ms_per_sweep": e0.elapsed_time(e1),
            "per_c": {str(c): {"status": nl.STATUS_NAMES[s["status"]], "newton": s["newton_iters"],
                               "final_rel_res": s["hist"][-1], "ms": s["t_total_ms"], **err_tp[str(c)]}
                      for c, s in stm.items()}}
    def alt_sweep(mode, **cfg):
        """The sweep with other handles (another configuration) on the same streams: one untimed
        pass, one timed."""
        hs = {c: nl.Solver(N_BENCH, c, stream=streams[c], lu_nb=args.lu_nb, lu_stream=args.lu_stream,
                           lu_lookahead=args.lu_lookahead, **cfg)
              for c in SWEEP}

        def run(c):
            try:
                hs[c].solve_device(xdev[c], tol=TOL, mode=mode)
            except nl.NLError:
                pass
            return hs[c].stats()

        for _ in range(2):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            futs = {c: pool.submit(run, c) for c in SWEEP}
            stc = {c: f.result() for c, f in futs.items()}
            e1.record()
            torch.cuda.synchronize()
        for h in hs.values():
            h.close()
        err = errors(None, stc)
        return {"ms_per_sweep": e0.elapsed_time(e1),
                "per_c": {str(c): {"status": nl.STATUS_NAMES[s["status"]], "newton": s["newton_iters"],
                                   "lin_iters": s["lin_iters"], "ms": s["t_total_ms"], "lin_ms": s["t_lin_ms"],
                                   **err[str(c)]}
                          for c, s in stc.items()}}

    # the binary16-arithmetic solve pair of the F16 step: a chain of 2N barrier steps in one CTA
    try:
        nl.kernel_timing("k_lusolve16h")
        one_tp(SWEEP[0], "F16")
        n16, ms16 = nl.kernel_timing(None)
        if n16:
            us = ms16 / n16 * 1e3
            fbytes = 2.0 * N_BENCH * N_BENCH  # both binary16 triangles
            extra["two_precision"]["F16"]["k_lusolve16h"] = {
                "launches": n16, "avg_us": us, "bound": "latency", "ns_per_barrier_step": us * 1e3 / (2 * N_BENCH),
                "factor_bytes_per_launch": fbytes, "achieved_GBps": fbytes / (us * 1e-6) / 1e9,
                "frac_of_hbm": fbytes / (us * 1e-6) / 1e9 / hbm_peak}
    except nl.NLError as e:
        extra["two_precision"]["F16"]["k_lusolve16h"] = {"error": str(e)}

    # interprecision ablation (Section 2.3): IR16 with the scaled binary16 correction of eq. (2.19)
    # against the on-the-fly correction of the "ir16" sweep above
    extra["ir16_scaled_half"] = alt_sweep("IR16", ir_variant=1)
    extra["ir16_scaled_half"]["note"] = "eq. (2.19): d = ||r|| fl32(U^-1 L^-1 fl16(r/||r||)), both solves in binary16"
    # GMRES-IR preconditioned with a single-precision copy of the binary16 factors (Section 2.3)
    extra["gmresir16_factors32"] = alt_sweep("GMRESIR16", gmres_factors32=1)
    extra["gmresir16_factors32"]["note"] = "the headline sweep with the factors promoted once per factorisation"
    # the optional scaling of J into the binary16 range (scale_fp16 = 1) against the unscaled headline sweep
    extra["gmresir16_scaled"] = alt_sweep("GMRESIR16", scale_fp16=1)
    extra["gmresir16_scaled"]["note"] = ("J_h = fl16(R J32), power-of-two row factors (2^12 here), solves applied to "
                                         "R v; against the unscaled headline sweep")
    extra["ir16_scaled"] = alt_sweep("IR16", scale_fp16=1)
    extra["sequential"] = {"ms_per_sweep": ms_seq[0], "solves_per_s": len(SWEEP) / (ms_seq[0] / 1e3),
                           "note": "the same five solves one after another on one stream"}
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16/f32/f64", "data": "synthetic (the paper's H-equation, x0=ones)",
            "config": {"workload": WORKLOAD, "N": N_BENCH, "c": list(SWEEP), "mode": "GMRESIR16",
                       "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{ws}",
                       "concurrency": "the five solves of a step on five streams (one host thread each)",
                       "cuda_device_max_connections": int(os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8"))},
            "roofline": roofline, "roofline_lu": roofline_lu, "kernels": kern, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
            "per_c": per_c, **extra}
    from paper_2307_16051_gb300 import workloads as W
    if not args.no_batch:
        line["batched"] = bench_batched(nl, W, torch, dev, args.steps, args.warmup, tc_peak, fp64=not args.no_fp64)
    if not args.no_large:
        line["large"] = bench_large(nl, torch, dev, hbm_peak, tc_peak, fp64=not args.no_large_fp64)
    if args.serve_seconds > 0:
        line["serving"] = bench_serving(nl, W, args.serve_seconds)
    if args.serve_fp64_seconds > 0:
        line["serving_fp64lu"] = bench_serving(nl, W, args.serve_fp64_seconds, mode="FP64LU", drain_s=30.0)
        line["serving_fp64lu"]["note"] = ("the same trace window as the three-precision server; FP64-LU Newton cannot "
                                          "keep up with 200 req/s, so the server is stopped 30 s after the last "
                                          "arrival and the requests still waiting then are counted as not served")
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample()
    if rank == 0:
        print(json.dumps(line), flush=True)
    for s in solvers.values():
        s.close()
    pool.shutdown()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
