"""Pins for the oracle's LU factorisations and triangular solves
(Section 1.3: Gaussian elimination; Section 2: half-precision factorisation;
Section 2.3, eqs. (2.16)-(2.19): solves with interprecision transfers).

Independent references:
  * exact rational Gaussian elimination with partial pivoting (fractions),
  * LAPACK getrf through scipy.linalg.lu_factor (a library run as a black box),
  * a binary16 / binary32 machine built from numpy's float16 / float32
    scalar arithmetic (each operation correctly rounded by numpy), written as
    plain Python loops for small N.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2307_16051_gb300 import workloads as W


def exact_gepp(A):
    """Gaussian elimination with partial pivoting in exact rationals."""
    n = len(A)
    a = [[Fraction(v) for v in row] for row in A]
    piv = []
    for k in range(n):
        p = max(range(k, n), key=lambda i: (abs(a[i][k]), -i))
        piv.append(p)
        a[k], a[p] = a[p], a[k]
        if a[k][k] == 0:
            continue
        for i in range(k + 1, n):
            a[i][k] /= a[k][k]
            for j in range(k + 1, n):
                a[i][j] -= a[i][k] * a[k][j]
    return a, piv


def has_exact_tie(A):
    n = len(A)
    a = [[Fraction(v) for v in row] for row in A]
    for k in range(n):
        mags = sorted((abs(a[i][k]) for i in range(k, n)), reverse=True)
        if len(mags) > 1 and mags[0] == mags[1]:
            return True
        p = max(range(k, n), key=lambda i: (abs(a[i][k]), -i))
        a[k], a[p] = a[p], a[k]
        if a[k][k] == 0:
            return True
        for i in range(k + 1, n):
            a[i][k] /= a[k][k]
            for j in range(k + 1, n):
                a[i][j] -= a[i][k] * a[k][j]
    return False


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_lu64_matches_exact_rational_elimination(n):
    g = np.random.default_rng(100 + n)
    done = 0
    while done < 4:
        A = g.integers(-9, 10, size=(n, n)).astype(np.float64)
        if has_exact_tie(A):
            continue
        ex, piv = exact_gepp(A.tolist())
        LU, ipiv, info = O.lu64(A)
        assert info == 0
        assert list(ipiv) == piv
        exf = np.array([[float(v) for v in row] for row in ex])
        assert np.allclose(LU, exf, rtol=1e-13, atol=1e-13)
        done += 1


def test_lu64_matches_lapack_getrf():
    for seed, n in [(1, 50), (2, 97), (3, 128)]:
        A = W.random_matrix(n, seed)
        LU, ipiv, info = O.lu64(A)
        lu_ref, piv_ref = scipy.linalg.lu_factor(A)
        assert info == 0
        assert np.array_equal(ipiv, piv_ref)
        assert np.max(np.abs(LU - lu_ref)) <= 1e-11 * np.max(np.abs(lu_ref))


def test_lu64_zero_pivot_reports_info():
    A = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [1.0, 1.0, 1.0]])
    A[:, 0] = 0.0  # first column all zero -> singular at step 1
    _, _, info = O.lu64(A)
    assert info == 1


def test_lusolve64_solves():
    A = W.random_matrix(60, 7)
    b = W.random_vector(60, 8)
    LU, ipiv, _ = O.lu64(A)
    x = O.lusolve64(LU, ipiv, b)
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b) * np.linalg.cond(A)


# ---------------------------------------------------------------- binary16 --

def np16_gepp(A16):
    """Gaussian elimination in numpy float16 scalar arithmetic: every
    division, product and difference rounded to binary16 by numpy."""
    a = np.array(A16, dtype=np.float16)
    n = a.shape[0]
    piv = []
    for k in range(n):
        col = np.abs(a[k:, k].astype(np.float64))
        p = k + int(np.argmax(col))  # first maximum
        piv.append(p)
        a[[k, p]] = a[[p, k]]
        if a[k, k] == 0:
            continue
        for i in range(k + 1, n):
            l = np.float16(a[i, k] / a[k, k])
            a[i, k] = l
            for j in range(k + 1, n):
                a[i, j] = np.float16(a[i, j] - np.float16(l * a[k, j]))
    return a.astype(np.float64), piv


def np16_gepp_recip(A16):
    """The same elimination with the column scaled by the rounded reciprocal
    of the pivot: r = fl16(1 / a_kk), l = fl16(a_ik r), in numpy float16."""
    a = np.array(A16, dtype=np.float16)
    n = a.shape[0]
    piv = []
    for k in range(n):
        col = np.abs(a[k:, k].astype(np.float64))
        p = k + int(np.argmax(col))
        piv.append(p)
        a[[k, p]] = a[[p, k]]
        if a[k, k] == 0:
            continue
        r = np.float16(np.float16(1.0) / a[k, k])
        for i in range(k + 1, n):
            l = np.float16(a[i, k] * r)
            a[i, k] = l
            for j in range(k + 1, n):
                a[i, j] = np.float16(a[i, j] - np.float16(l * a[k, j]))
    return a.astype(np.float64), piv


@pytest.mark.parametrize("n,seed", [(4, 1), (9, 2), (13, 3), (16, 4)])
def test_lu16_recip_bit_exact_vs_numpy_float16_machine(n, seed):
    A = W.random_matrix(n, seed).astype(np.float16).astype(np.float64)
    ref, piv = np16_gepp_recip(A)
    LU, ipiv, info, ovf = O.lu16_recip(A)
    assert not ovf and list(ipiv) == piv
    assert np.array_equal(LU, ref)
    # and it is a different elimination from the quotient one
    LUq, _, _, _ = O.lu16(A)
    assert not np.array_equal(LU, LUq) or n <= 4


@pytest.mark.parametrize("n,seed", [(4, 1), (9, 2), (13, 3), (16, 4)])
def test_lu16_bit_exact_vs_numpy_float16_machine(n, seed):
    A = W.random_matrix(n, seed).astype(np.float16).astype(np.float64)
    ref, piv = np16_gepp(A)
    LU, ipiv, info, ovf = O.lu16(A)
    assert not ovf
    assert list(ipiv) == piv
    assert np.array_equal(LU, ref)


def test_lu16_with_subnormals_bit_exact():
    # entries around the binary16 subnormal range (the paper's Jacobian at
    # large N has many off-diagonal entries below 2^-14)
    g = np.random.default_rng(5)
    n = 12
    A = g.standard_normal((n, n)) * 2.0 ** -16
    A[np.arange(n), np.arange(n)] = 1.0 + g.uniform(0, 1, n)
    A = A.astype(np.float16).astype(np.float64)
    ref, piv = np16_gepp(A)
    LU, ipiv, _, _ = O.lu16(A)
    assert list(ipiv) == piv and np.array_equal(LU, ref)


def test_lu16_values_are_binary16_and_backward_stable():
    A, perm = W.pivot_forcing_matrix(120, 11)
    A16 = O.fl16(A)
    LU, ipiv, info, ovf = O.lu16(A16)
    assert info == 0 and not ovf
    assert np.array_equal(O.fl16(LU), LU)
    # the pivot sequence of a strongly dominant, permuted matrix is unique
    _, ipiv64, _ = O.lu64(A16)
    assert np.array_equal(ipiv, ipiv64)
    n = A.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    PA = A16.copy()
    for k, p in enumerate(ipiv):
        PA[[k, p]] = PA[[p, k]]
    err = np.max(np.abs(PA - L @ U)) / np.max(np.abs(A16))
    assert err <= 4 * n * 2.0 ** -11


def test_lu32_matches_numpy_float32_machine():
    n = 10
    A = W.random_matrix(n, 21).astype(np.float32)
    a = A.copy()
    piv = []
    for k in range(n):
        p = k + int(np.argmax(np.abs(a[k:, k])))
        piv.append(p)
        a[[k, p]] = a[[p, k]]
        for i in range(k + 1, n):
            l = np.float32(a[i, k] / a[k, k])
            a[i, k] = l
            for j in range(k + 1, n):
                a[i, j] = np.float32(a[i, j] - np.float32(l * a[k, j]))
    LU, ipiv, _ = O.lu32(A)
    assert list(ipiv) == piv and np.array_equal(LU, a)


def _apply_piv(v, ipiv):
    v = v.copy()
    for k, p in enumerate(ipiv):
        v[[k, p]] = v[[p, k]]
    return v


def test_lusolve_fly_bit_exact_vs_float32_machine():
    """Eq. (2.16): binary16 factors promoted to single, single arithmetic."""
    n = 14
    A16 = O.fl16(W.random_matrix(n, 31))
    LU, ipiv, _, _ = O.lu16(A16)
    b = W.random_vector(n, 32).astype(np.float32)
    y = _apply_piv(b, ipiv)
    for i in range(n):
        s = y[i]
        for t in range(i):
            s = np.float32(s - np.float32(np.float32(LU[i, t]) * y[t]))
        y[i] = s
    for i in reversed(range(n)):
        s = y[i]
        for t in range(i + 1, n):
            s = np.float32(s - np.float32(np.float32(LU[i, t]) * y[t]))
        y[i] = np.float32(s / np.float32(LU[i, i]))
    assert np.array_equal(O.lusolve_fly(LU, ipiv, b), y)


def test_lusolve16_bit_exact_vs_float16_machine():
    """Inner solve of eqs. (2.17) and (2.19) and the F16 step: all in
    binary16, the back substitution taking row i's terms from the last
    column down."""
    n = 14
    A16 = O.fl16(W.random_matrix(n, 41))
    LU, ipiv, _, _ = O.lu16(A16)
    b = O.fl16(W.random_vector(n, 42) / 4)
    y = _apply_piv(b, ipiv).astype(np.float16)
    L16 = LU.astype(np.float16)
    for i in range(n):
        s = y[i]
        for t in range(i):
            s = np.float16(s - np.float16(L16[i, t] * y[t]))
        y[i] = s
    for i in reversed(range(n)):
        s = y[i]
        for t in reversed(range(i + 1, n)):
            s = np.float16(s - np.float16(L16[i, t] * y[t]))
        y[i] = np.float16(s / L16[i, i])
    assert np.array_equal(O.lusolve16(LU, ipiv, b), y.astype(np.float64))


def test_lusolve_fly_accuracy_on_pivoted_matrix():
    A, _ = W.pivot_forcing_matrix(200, 51)
    A16 = O.fl16(A)
    LU, ipiv, _, _ = O.lu16(A16)
    xtrue = W.random_vector(200, 52)
    b = (A16 @ xtrue).astype(np.float32)
    x = O.lusolve_fly(LU, ipiv, b).astype(np.float64)
    # the factors are those of a binary16 perturbation of A: error O(u_h)
    assert np.linalg.norm(x - xtrue) / np.linalg.norm(xtrue) <= 50 * 2.0 ** -11


def np_lu16_dev(A16, nb):
    """Binary16 storage / binary32 arithmetic elimination written with numpy
    float32 and float16 scalars: pivot rows and multipliers rounded to
    binary16 when formed, the remaining submatrix rounded to binary16 after
    every nb steps."""
    a = np.array(A16, dtype=np.float32)
    n = a.shape[0]
    piv = []
    for k in range(n):
        p = k + int(np.argmax(np.abs(a[k:, k])))
        piv.append(p)
        a[[k, p]] = a[[p, k]]
        a[k, k:] = a[k, k:].astype(np.float16).astype(np.float32)
        if a[k, k] != 0:
            for i in range(k + 1, n):
                l = np.float32(np.float16(np.float32(a[i, k] / a[k, k])))
                a[i, k] = l
                for j in range(k + 1, n):
                    a[i, j] = np.float32(a[i, j] - np.float32(l * a[k, j]))
        if (k + 1) % nb == 0 or k == n - 1:
            a[k + 1:, k + 1:] = a[k + 1:, k + 1:].astype(np.float16).astype(np.float32)
    return a.astype(np.float64), piv


@pytest.mark.parametrize("n,nb,seed", [(7, 1, 1), (10, 3, 2), (16, 4, 3), (17, 8, 4), (12, 64, 5)])
def test_lu16_dev_bit_exact_vs_numpy_machine(n, nb, seed):
    A = O.fl16(W.random_matrix(n, seed))
    ref, piv = np_lu16_dev(A, nb)
    LU, ipiv, info, ovf = O.lu16_dev(A, nb)
    assert info == 0 and not ovf
    assert list(ipiv) == piv
    assert np.array_equal(LU, ref)


def test_lu16_dev_accuracy_beats_per_op_binary16():
    """Carrying the unfinished submatrix in binary32 keeps the small updates
    that per-operation binary16 rounding drops (Section 2.2 discusses how the
    accuracy of the half-precision factors drives IR convergence)."""
    N, c = 600, 0.99
    from oracle import oracle as OO
    x = np.ones(N)
    J = OO.jacobian(N, c, x)
    J16 = OO.fl16(J.astype(np.float32).astype(np.float64))
    res = {}
    for name, (LU, ipiv, info, ovf) in (("dev", OO.lu16_dev(J16, 64)), ("op", OO.lu16(J16))):
        L = np.tril(LU, -1) + np.eye(N)
        U = np.triu(LU)
        res[name] = np.linalg.norm(J16 - L @ U, 2)  # no pivoting occurs here
        assert list(ipiv) == list(range(N))
    assert res["dev"] < res["op"] / 3
    assert res["dev"] <= 4 * 2.0 ** -11


def test_uniform_power_of_two_scaling_changes_no_rounding():
    """Scaling a matrix by 2^k commutes with every binary16 and binary32
    rounding as long as no result is subnormal or overflows: the factors of
    fl16(2^k A) are those of fl16(A) with U multiplied by 2^k and the same L,
    and IR with the row factors applied to the right side returns the same
    u bit for bit (the scaled solve multiplies each right side by 2^k, which
    the factors' U undoes exactly)."""
    n, k = 48, 10
    g = np.random.default_rng(11)
    A = np.eye(n) * 4.0 + g.uniform(0.25, 1.0, (n, n)) * np.where(g.random((n, n)) < 0.5, -1.0, 1.0)
    A16 = O.fl16(A)
    LU, ipiv, _, _ = O.lu16_dev(A16, 16)
    tiny = (np.abs(LU) < 2.0 ** -14) & (LU != 0)
    assert not tiny.any()  # the premise: no subnormal factor entry
    LUs, ipivs, _, _ = O.lu16_dev(O.fl16(A16 * 2.0 ** k), 16)
    assert np.array_equal(ipiv, ipivs)
    L = np.tril(LU, -1)
    assert np.array_equal(np.tril(LUs, -1), L)
    assert np.array_equal(np.triu(LUs), np.triu(LU) * 2.0 ** k)
    A32 = A16.astype(np.float32)
    b = g.standard_normal(n).astype(np.float32)
    for solver in (O.SOLVER_IR_FLY, O.SOLVER_GMRES):
        u0, st0 = O.linsolve(A32, LU, ipiv, b, solver=solver, eta=1e-6)
        u1, st1 = O.linsolve(A32, LUs, ipivs, b, solver=solver, eta=1e-6, rs=np.full(n, 2.0 ** k))
        assert np.array_equal(u0, u1) and st0 == st1
