"""Command-line front end: solve the H-equation once (or a few times) on the
GPU and print the solver statistics as JSON.

    python -m paper_2307_16051_gb300 --N 4096 --c 0.99 --mode GMRESIR16 --repeat 2
    python -m paper_2307_16051_gb300 --N 4096 --c 0.99 --mode F16 --lu16-arith 1 --newton-maxit 10 --tol 1e-9
    python -m paper_2307_16051_gb300 --batch 512 --repeat 2          # the batched workload
    python -m paper_2307_16051_gb300 --batch 512 --batch-nrange 1025 2048 --lu-nb 64 --trailing-gemm 5 --task-times
    python -m paper_2307_16051_gb300 --serve-seconds 2               # the serving trace
"""
import argparse
import json

from . import nl


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--c", type=float, default=0.99)
    ap.add_argument("--mode", default=None, choices=sorted(nl.MODES))
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--repeat", type=int, default=1, help="solves on the same handle (the last one is reported)")
    ap.add_argument("--eta", type=float, default=1e-4)
    ap.add_argument("--lu-nb", type=int, default=0)
    ap.add_argument("--newton-maxit", type=int, default=30)
    ap.add_argument("--ir-variant", type=int, default=0, choices=[0, 1],
                    help="1: IR with the scaled binary16 correction of eq. (2.19)")
    ap.add_argument("--gmres-factors32", type=int, default=0, choices=[0, 1],
                    help="1: GMRES-IR preconditioned with a single-precision copy of the factors")
    ap.add_argument("--lu16-arith", type=int, default=0, choices=[0, 1],
                    help="1: the half-precision factorisation with every operation in binary16")
    ap.add_argument("--scale-fp16", type=int, default=0, choices=[0, 1],
                    help="1: J scaled into the binary16 range (power-of-two row factors) before the down-cast")
    ap.add_argument("--fft-f", type=int, default=0, choices=[-1, 0, 1],
                    help="F by the FFT convolution (1), the direct sum (-1), or the automatic choice (0)")
    ap.add_argument("--batch", type=int, default=0,
                    help="solve the first BATCH instances of the batched workload (N log-uniform in [64, 2048], "
                         "c uniform in [0.1, 0.999], seed 230716051) together")
    ap.add_argument("--batch-nrange", type=int, nargs=2, default=None, metavar=("NMIN", "NMAX"),
                    help="keep only the batch instances with NMIN <= N <= NMAX")
    ap.add_argument("--trailing-gemm", type=int, default=0, choices=[0, 1, 2, 3, 4, 5],
                    help="batch grouped-LU update with --lu-nb: 1 SIMT, 2 tcgen05 (three launches per outer step), "
                         "3 / 4 / 5 one persistent launch (SIMT 64x64, SIMT 128x64, tcgen05 128x128)")
    ap.add_argument("--task-times", action="store_true",
                    help="batch: report the persistent grouped LU's per-task times over the factorisations timed "
                         "at creation")
    ap.add_argument("--serve-seconds", type=float, default=0.0,
                    help="replay the first SECONDS of the serving trace (Poisson 200/s) through the request loop")
    args = ap.parse_args()
    if args.batch > 0:
        from . import workloads as W
        inst = W.batch_instances()[: args.batch]
        if args.batch_nrange:
            inst = [(n, c) for n, c in inst if args.batch_nrange[0] <= n <= args.batch_nrange[1]]
        if args.task_times:
            nl.grouped_task_times(True)
        with nl.Batch([n for n, _ in inst], [c for _, c in inst], eta_j=args.eta, lu_nb=args.lu_nb,
                      trailing_gemm=args.trailing_gemm) as B:
            times = nl.grouped_task_times(False) if args.task_times else None
            for _ in range(max(1, args.repeat)):
                xs, status = B.solve(tol=args.tol, mode=args.mode or "IR16_GMRES")
            info = B.info()
        if times is not None:
            info["task_times"] = times
        info["status_name"] = nl.STATUS_NAMES[status]
        print(json.dumps(info))
        return
    if args.serve_seconds > 0:
        from . import workloads as W
        trace = W.serving_trace(duration_s=args.serve_seconds)
        with nl.Server(mode=args.mode or "IR16_GMRES", tol=args.tol) as S:
            for t, N, c in trace:
                S.submit(N, c, arrival_s=t)
            S.start()
            S.drain(600.0)
            print(json.dumps(S.info()))
        return
    with nl.Solver(args.N, args.c, eta_j=args.eta, lu_nb=args.lu_nb, newton_maxit=args.newton_maxit,
                   ir_variant=args.ir_variant, gmres_factors32=args.gmres_factors32, lu16_arith=args.lu16_arith,
                   scale_fp16=args.scale_fp16, fft_f=args.fft_f) as s:
        for _ in range(max(1, args.repeat)):
            x, status = s.solve(tol=args.tol, mode=args.mode or "GMRESIR16")
        st = s.stats()
    st["status_name"] = nl.STATUS_NAMES[status]
    st["x_min"], st["x_max"] = float(x.min()), float(x.max())
    print(json.dumps(st))


if __name__ == "__main__":
    main()
