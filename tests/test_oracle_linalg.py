"""Pins of the oracle's vector operations and dense LU.

Vector ops (Sec. 4 streaming / reduction operations) are checked against their
definitions evaluated independently (numpy elementwise, exactly rounded sums
via math.fsum).  The LU is checked against exact rational solutions of small
integer systems (fractions.Fraction Gauss-Jordan), its pivot tie-break, its
zero-pivot report, and the normwise backward error on random blocks.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2011_12984_b300 import gen


def test_streaming_ops_match_elementwise_definition():
    x, y, w, v = gen.uniform_vectors(1000, 4, seed=7)
    assert np.array_equal(oracle.linear_sum(0.3, x, -1.7, y), 0.3 * x + (-1.7) * y)
    c = np.array([0.5, -2.0, 3.0])
    z = oracle.linear_combination(c, [x, y, w])
    ref = np.array([math.fsum([c[0] * x[i], c[1] * y[i], c[2] * w[i]]) for i in range(1000)])
    scale = np.abs(c[0] * x) + np.abs(c[1] * y) + np.abs(c[2] * w)
    assert np.all(np.abs(z - ref) <= 4e-16 * scale)
    a = np.array([2.0, -0.25])
    zs = oracle.scale_add_multi(a, x, [y, w])
    assert np.array_equal(zs[0], 2.0 * x + y) and np.array_equal(zs[1], -0.25 * x + w)


def test_reductions_match_exactly_rounded_sums():
    x, y, w = gen.uniform_vectors(20001, 3, seed=11)
    d, s = oracle.dot_prod_multi(x, [y, w, x])
    for j, v in enumerate([y, w, x]):
        exact = math.fsum((x * v).tolist())
        assert abs(d[j] - exact) <= 2e-16 * np.sum(np.abs(x * v))
        assert abs(s[j] - np.sum(np.abs(x * v))) <= 1e-12 * s[j]
    ewt = 1.0 / (1e-4 * np.abs(y) + 1e-8)
    nrm = oracle.wrms_norm(x, ewt)
    exact = math.sqrt(math.fsum(((x * ewt) ** 2).tolist()) / x.size)
    assert abs(nrm - exact) <= 4e-16 * exact
    assert oracle.wrms_norm(np.zeros(5), np.ones(5)) == 0.0


def frac_solve(A, b):
    n = len(b)
    M = [[Fraction(int(A[i][j])) for j in range(n)] + [Fraction(int(b[i]))] for i in range(n)]
    for k in range(n):
        p = next(i for i in range(k, n) if M[i][k] != 0)
        M[k], M[p] = M[p], M[k]
        for i in range(n):
            if i != k and M[i][k] != 0:
                f = M[i][k] / M[k][k]
                M[i] = [a - f * c for a, c in zip(M[i], M[k])]
    return [M[i][n] / M[i][i] for i in range(n)]


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_lu_solves_small_integer_systems_exactly(n):
    rng = np.random.default_rng(n)
    for _ in range(20):
        A = rng.integers(-9, 10, size=(n, n)).astype(float)
        if abs(np.linalg.det(A)) < 0.5:
            continue
        b = rng.integers(-9, 10, size=n).astype(float)
        lu, piv, info = oracle.lu_factor(A)
        assert info == 0
        x = oracle.lu_solve(lu, piv, b)
        ex = np.array([float(v) for v in frac_solve(A, b)])
        assert np.all(np.abs(x - ex) <= 1e-12 * np.maximum(1.0, np.abs(ex)))


def test_lu_pivot_tie_break_and_zero_pivot():
    _, piv, info = oracle.lu_factor(np.array([[1.0, 2.0], [-1.0, 3.0]]))
    assert info == 0 and piv[0] == 0           # |1| == |-1|: lowest row kept
    _, piv, info = oracle.lu_factor(np.array([[0.0, 1.0], [2.0, 0.0]]))
    assert info == 0 and piv[0] == 1
    _, piv, info = oracle.lu_factor(np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [1.0, 0.0, 1.0]]))
    assert info == 3                           # exactly singular: zero pivot at step 2


@pytest.mark.parametrize("n", [3, 10, 32, 54])
def test_lu_backward_error(n):
    rng = np.random.default_rng(100 + n)
    J = rng.standard_normal((n, n)) * 10.0 ** rng.uniform(-2, 6, size=(n, n))
    M = np.eye(n) - 1e-3 * J
    b = rng.standard_normal(n)
    lu, piv, info = oracle.lu_factor(M)
    x = oracle.lu_solve(lu, piv, b)
    r = M @ x - b
    eta = np.max(np.abs(r)) / (np.max(np.sum(np.abs(M), axis=1)) * np.max(np.abs(x)) + np.max(np.abs(b)))
    assert eta <= 1e-14


def test_support_ops_fixed_points():
    """Values the definitions fix exactly: scaling by 1 and 0, constants,
    |x| of signed values, 1/x of powers of two, x + 0, and error weights of
    y = 0 (1/atol) and of powers of two with atol = 0.5 ulp-free choices."""
    x = np.array([-3.5, -0.0, 0.0, 2.0, 1e300, -1e-300])
    assert np.array_equal(oracle.scale(1.0, x), x)
    assert np.all(oracle.scale(0.0, x[np.isfinite(x)]) == 0.0)
    assert np.array_equal(oracle.const(7.25, 5), np.full(5, 7.25))
    assert np.array_equal(oracle.abs_(x), np.array([3.5, 0.0, 0.0, 2.0, 1e300, 1e-300]))
    p2 = 2.0 ** np.arange(-20, 21)
    assert np.array_equal(oracle.inv(p2), 2.0 ** -np.arange(-20, 21))
    assert np.array_equal(oracle.inv(-p2), -(2.0 ** -np.arange(-20, 21)))
    assert np.array_equal(oracle.add_const(x[:4], 0.0), x[:4] + 0.0)
    assert np.array_equal(oracle.add_const(np.array([1.0, 2.0]), 0.5), np.array([1.5, 2.5]))
    w = oracle.error_weights(0.25, 0.5, np.array([0.0, 2.0, -2.0, 6.0]))
    assert np.array_equal(w, np.array([2.0, 1.0, 1.0, 0.5]))      # 1/(0.25*|y| + 0.5)
