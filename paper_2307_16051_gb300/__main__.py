"""Command-line front end: solve the H-equation once (or a few times) on the
GPU and print the solver statistics as JSON.

    python -m paper_2307_16051_gb300 --N 4096 --c 0.99 --mode GMRESIR16 --repeat 2
"""
import argparse
import json

from . import nl


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--c", type=float, default=0.99)
    ap.add_argument("--mode", default="GMRESIR16", choices=sorted(nl.MODES))
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--repeat", type=int, default=1, help="solves on the same handle (the last one is reported)")
    ap.add_argument("--eta", type=float, default=1e-4)
    ap.add_argument("--lu-nb", type=int, default=0)
    args = ap.parse_args()
    with nl.Solver(args.N, args.c, eta_j=args.eta, lu_nb=args.lu_nb) as s:
        for _ in range(max(1, args.repeat)):
            x, status = s.solve(tol=args.tol, mode=args.mode)
        st = s.stats()
    st["status_name"] = nl.STATUS_NAMES[status]
    st["x_min"], st["x_max"] = float(x.min()), float(x.max())
    print(json.dumps(st))


if __name__ == "__main__":
    main()
