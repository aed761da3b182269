"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module holds no arithmetic of the method: it only draws numbers.  The
paper's test problem (Section 3, eq. (3.2)) is fully determined by N, c and
x0 = ones, so the nonlinear workloads below are lists of (N, c) pairs; the
matrix generators feed the kernel-level LU / triangular-solve parity tests.
"""
from __future__ import annotations

import math

import numpy as np

# conditioning sweep of the paper's example (Tables 2-3 use c = .99, .9999)
SWEEP_C = (0.5, 0.9, 0.99, 0.9999, 0.999999)


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_matrix(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Dense n x n float64 matrix with i.i.d. N(0, scale^2) entries."""
    return rng(seed).standard_normal((n, n)) * scale


def pivot_forcing_matrix(n: int, seed: int, margin: float = 4.0) -> tuple[np.ndarray, np.ndarray]:
    """A = P B with B strongly diagonally dominant (|b_jj| >= margin * sum of
    |b_ij|, i != j, over column j) and P a random row permutation.

    Partial pivoting on A must then pick, at step j, the row that holds b_j,
    with a wide gap to the runner-up, so the pivot sequence is unique and
    insensitive to rounding.  Returns (A, perm) with A[i] = B[perm[i]]."""
    g = rng(seed)
    B = g.uniform(-1.0, 1.0, size=(n, n))
    np.fill_diagonal(B, 0.0)
    colsum = np.abs(B).sum(axis=0)
    d = (margin * colsum + 1.0) * g.choice([-1.0, 1.0], size=n) * g.uniform(1.0, 2.0, size=n)
    B[np.arange(n), np.arange(n)] = d
    perm = g.permutation(n)
    return B[perm], perm


def random_vector(n: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(n)


def batch_instances(count: int = 512, seed: int = 230716051, n_lo: int = 64, n_hi: int = 2048,
                    c_lo: float = 0.1, c_hi: float = 0.999) -> list[tuple[int, float]]:
    """Independent problem instances for the batched path: N log-uniform in
    [n_lo, n_hi] (rounded), c uniform in [c_lo, c_hi]."""
    g = rng(seed)
    Ns = np.rint(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(int)
    cs = g.uniform(c_lo, c_hi, size=count)
    return [(int(n), float(c)) for n, c in zip(Ns, cs)]


def serving_trace(seed: int = 16051, rate_per_s: float = 200.0, duration_s: float = 60.0,
                  sizes=(256, 1024, 4096, 16384), probs=(0.5, 0.3, 0.15, 0.05),
                  c_lo: float = 0.5, c_hi: float = 0.9999) -> list[tuple[float, int, float]]:
    """Poisson arrival trace: (arrival time in s, N, c), sorted by time."""
    g = rng(seed)
    out = []
    t = 0.0
    while True:
        t += g.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        n = int(g.choice(sizes, p=probs))
        c = float(g.uniform(c_lo, c_hi))
        out.append((t, n, c))
    return out
