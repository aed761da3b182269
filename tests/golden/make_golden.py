"""Write tests/golden/sweep_n4096.json: oracle results for the conditioning
sweep of the paper's example (Section 3, eq. (3.2)) at N = 4096, used by the
GPU parity tests at full size.

Calls only the CPU oracle.  For every c in {.5, .9, .99, .9999, .999999} and
every mode (FP64LU, IR16, GMRESIR16; eta_J = 1e-4, restart 30, inner tol
1e-4, half-precision LU with binary32 arithmetic and rounding period 128) it
stores the Newton and linear iteration counts, the residual history, and the
FP64-LU solution at 64 seeded sample indices plus its sum.

It also writes sweep_n4096_x.npy: the full FP64-LU oracle solution for each
c of the sweep (float64, shape 5 x 4096, rows in the order of SWEEP), which
the GPU tests compare element by element and the benchmark uses to state
each result's error against the FP64 oracle.

Usage: python tests/golden/make_golden.py          (about 15-30 minutes on 8 cores)
       python tests/golden/make_golden.py --x-only (the solutions only)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import oracle as O  # noqa: E402

N = 4096
SWEEP = (0.5, 0.9, 0.99, 0.9999, 0.999999)
SAMPLE = sorted(set(np.random.default_rng(4096).choice(N, 62, replace=False).tolist() + [0, N - 1]))


HERE = os.path.dirname(os.path.abspath(__file__))


def write_solutions(out=os.path.join(HERE, "sweep_n4096_x.npy")):
    xs = np.empty((len(SWEEP), N))
    for k, c in enumerate(SWEEP):
        t = time.time()
        x, r = O.newton(N, c, "FP64LU", tol=1e-10, lu_nb=128)
        assert r["status"] == 0
        xs[k] = x
        print(c, "FP64LU", r["newton_iters"], "%.1fs" % (time.time() - t), flush=True)
    np.save(out, xs)


def main(out=os.path.join(HERE, "sweep_n4096.json")):
    res = {"N": N, "tol": 1e-10, "eta": 1e-4, "lu_nb": 128, "sample_idx": SAMPLE, "oracle_threads": O.num_threads(),
           "cases": {}}
    for c in SWEEP:
        for mode in ("FP64LU", "IR16", "GMRESIR16"):
            t = time.time()
            x, r = O.newton(N, c, mode, tol=1e-10, lu_nb=128)
            r["seconds"] = time.time() - t
            r["x_sample"] = [float(x[i]) for i in SAMPLE]
            r["x_sum"] = float(x.sum())
            r["moment"] = float(c / (2 * N) * x.sum())
            res["cases"][f"{c}/{mode}"] = r
            print(c, mode, r["status"], r["newton_iters"], r["lin_iters"], "%.1fs" % r["seconds"], flush=True)
    with open(out, "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    if "--x-only" not in sys.argv:
        main()
    write_solutions()
