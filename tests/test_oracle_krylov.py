"""Pins for the oracle's IR and GMRES-IR (Section 2.2, Algorithm IR and the
left-preconditioned GMRES-IR; termination rules of Section 3.1)."""
import numpy as np

from oracle import oracle as O
from paper_2307_16051_gb300 import workloads as W


def _system(n, seed, cond_boost=0.0):
    A, _ = W.pivot_forcing_matrix(n, seed, margin=1.0)
    A = A + cond_boost * np.outer(W.random_vector(n, seed + 1), W.random_vector(n, seed + 2))
    A32 = A.astype(np.float32)
    LU, ipiv, info, ovf = O.lu16(O.fl16(A32.astype(np.float64)))
    assert info == 0 and not ovf
    return A32, LU, ipiv


def _precond(LU, ipiv, v):
    return O.lusolve_fly(LU, ipiv, v.astype(np.float32)).astype(np.float64)


def test_gmres_minimises_preconditioned_residual_over_krylov_space():
    """For j Arnoldi steps (one cycle, tolerance 0) the GMRES iterate solves
    min ||M^{-1}(r - A d)|| over d in K_j(M^{-1}A, M^{-1}r): compare the
    attained residual with a dense least-squares solve on an explicitly
    built (orthonormalised) Krylov basis."""
    n = 80
    A32, LU, ipiv = _system(n, 3, cond_boost=0.3)
    A = A32.astype(np.float64)
    r = W.random_vector(n, 4)
    z0 = _precond(LU, ipiv, r)
    for j in (1, 2, 3, 5, 8):
        d, steps = O.gmres(A32, LU, ipiv, r, m=j, tol=0.0, cycles=1)
        assert steps == j
        # Krylov basis of the same operator, Householder-orthonormalised
        K = [z0 / np.linalg.norm(z0)]
        for _ in range(j - 1):
            w = _precond(LU, ipiv, A @ K[-1])
            K.append(w / np.linalg.norm(w))
        Q, _ = np.linalg.qr(np.array(K).T)
        MA = np.array([_precond(LU, ipiv, A @ Q[:, i]) for i in range(j)]).T
        y, *_ = np.linalg.lstsq(MA, z0, rcond=None)
        best = np.linalg.norm(z0 - MA @ y)
        got = np.linalg.norm(z0 - np.array([_precond(LU, ipiv, A @ d)]).ravel())
        assert abs(got - best) <= 1e-5 * np.linalg.norm(z0) + 1e-3 * best


def test_full_gmres_solves_system():
    n = 60
    A32, LU, ipiv = _system(n, 5, cond_boost=0.5)
    r = W.random_vector(n, 6)
    d, steps = O.gmres(A32, LU, ipiv, r, m=n, tol=1e-10, cycles=3)
    A = A32.astype(np.float64)
    assert np.linalg.norm(A @ d - r) <= 1e-5 * np.linalg.norm(r)
    assert steps <= n + 5


def test_gmres_restarts_count_steps():
    n = 70
    A32, LU, ipiv = _system(n, 7, cond_boost=2.0)
    r = W.random_vector(n, 8)
    d1, s1 = O.gmres(A32, LU, ipiv, r, m=3, tol=1e-8, cycles=50)
    assert s1 % 3 == 0 or s1 < 150  # whole cycles unless converged mid-cycle
    A = A32.astype(np.float64)
    z = _precond(LU, ipiv, r - A @ d1)
    assert np.linalg.norm(z) <= 1e-6 * np.linalg.norm(_precond(LU, ipiv, r)) + 1e-7


def test_ir_converges_and_counts_corrections():
    n = 100
    A32, LU, ipiv = _system(n, 9)
    b = W.random_vector(n, 10).astype(np.float32)
    u, st = O.linsolve(A32, LU, ipiv, b, solver=O.SOLVER_IR_FLY, eta=1e-6, maxit=20)
    assert st["converged"] == 1 and st["failed"] == 0
    assert st["iters"] == st["outer"] >= 1
    A = A32.astype(np.float64)
    rel = np.linalg.norm(b - A @ u.astype(np.float64)) / np.linalg.norm(b)
    assert rel <= 1e-6 and abs(rel - st["relres"]) <= 1e-7
    # Algorithm IR closed form: after k corrections from u0 = 0 with exact
    # arithmetic the error contracts by the iteration matrix I - (LU)^{-1}A;
    # here the factors are within u_h of A, so each step gains ~3 digits
    assert st["iters"] <= 4


def test_ir_cheap_variant_converges():
    n = 100
    A32, LU, ipiv = _system(n, 9)
    b = W.random_vector(n, 10).astype(np.float32)
    u, st = O.linsolve(A32, LU, ipiv, b, solver=O.SOLVER_IR_CHEAP, eta=1e-5, maxit=20)
    assert st["converged"] == 1


def test_ir_failure_rule_returns_best_iterate():
    """Section 3.1: failure when the residual norm increases; the iterate
    with the best residual is returned."""
    n = 60
    g = np.random.default_rng(12)
    # ill-conditioned: the binary16 factors are far from A, IR diverges
    U, _ = np.linalg.qr(g.standard_normal((n, n)))
    V, _ = np.linalg.qr(g.standard_normal((n, n)))
    A = (U * np.logspace(0, -5, n)) @ V.T
    A32 = A.astype(np.float32)
    LU, ipiv, info, ovf = O.lu16(O.fl16(A32.astype(np.float64)))
    b = W.random_vector(n, 13).astype(np.float32)
    u, st = O.linsolve(A32, LU, ipiv, b, solver=O.SOLVER_IR_FLY, eta=1e-6, maxit=20)
    assert st["failed"] == 1 and st["converged"] == 0
    # recompute the residual history with growing caps: the returned iterate
    # has the smallest residual seen before the increase
    rels = []
    for k in range(1, st["outer"] + 1):
        uk, sk = O.linsolve(A32, LU, ipiv, b, solver=O.SOLVER_IR_FLY, eta=0.0, maxit=k)
        rels.append(np.linalg.norm(b - A32.astype(np.float64) @ uk.astype(np.float64)) / np.linalg.norm(b))
    final = np.linalg.norm(b - A32.astype(np.float64) @ u.astype(np.float64)) / np.linalg.norm(b)
    assert abs(final - min(rels)) <= 1e-6 * min(rels)
