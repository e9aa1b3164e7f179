"""Pins of the oracle's 1D rules, Lagrange bases and SBP operators (§3.1.3, eq. euler-sbp).

Each value is fixed independently of the oracle: closed forms of the GLL and
Gauss rules, numpy's Gauss-Legendre routine, and the exactness of derivative
matrices on polynomials.
"""
import math

import numpy as np
import pytest

import oracle


def test_gll_closed_forms():
    x, w = oracle.rule("gll", 0)
    assert list(x) == [0.0] and list(w) == [2.0]
    x, w = oracle.rule("gll", 1)
    np.testing.assert_allclose(x, [-1, 1], atol=0)
    np.testing.assert_allclose(w, [1, 1], rtol=1e-15)
    x, w = oracle.rule("gll", 2)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-16)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-15)
    x, w = oracle.rule("gll", 3)
    s = 1 / math.sqrt(5)
    np.testing.assert_allclose(x, [-1, -s, s, 1], rtol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-15)
    x, w = oracle.rule("gll", 4)
    s = math.sqrt(3 / 7)
    np.testing.assert_allclose(x, [-1, -s, 0, s, 1], rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=1e-14)


def test_gauss_closed_forms():
    x, w = oracle.rule("gauss", 0)
    np.testing.assert_allclose(x, [0.0], atol=0)
    np.testing.assert_allclose(w, [2.0], rtol=1e-15)
    x, w = oracle.rule("gauss", 1)
    s = 1 / math.sqrt(3)
    np.testing.assert_allclose(x, [-s, s], rtol=1e-15)
    np.testing.assert_allclose(w, [1, 1], rtol=1e-15)
    x, w = oracle.rule("gauss", 2)
    s = math.sqrt(3 / 5)
    np.testing.assert_allclose(x, [-s, 0, s], rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(w, [5 / 9, 8 / 9, 5 / 9], rtol=1e-15)


@pytest.mark.parametrize("r", range(0, 8))
def test_gauss_matches_numpy(r):
    x, w = oracle.rule("gauss", r)
    xn, wn = np.polynomial.legendre.leggauss(r + 1)
    np.testing.assert_allclose(x, xn, rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, wn, rtol=2e-14)


@pytest.mark.parametrize("r", range(1, 8))
def test_gll_interior_are_roots_of_dPr(r):
    x, w = oracle.rule("gll", r)
    dP = np.polynomial.legendre.Legendre.basis(r).deriv()
    roots = np.sort(dP.roots().real)
    np.testing.assert_allclose(x[1:-1], roots, atol=1e-14)
    # exactness of the GLL rule up to degree 2r-1
    for k in range(2 * r):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_sbp_and_derivative_exactness(p):
    x, w = oracle.rule("gll", p)
    n = p + 1
    D = np.array([[oracle.lagrange(x, j, x[i], deriv=True) for j in range(n)] for i in range(n)])
    Q = np.diag(w) @ D
    B = np.zeros((n, n))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(Q + Q.T, B, atol=2e-14)
    for k in range(p + 1):
        np.testing.assert_allclose(D @ x ** k, k * x ** max(k - 1, 0) if k else 0 * x, atol=1e-13)


def test_lagrange_cardinal():
    x, _ = oracle.rule("gauss", 3)
    for j in range(4):
        for i in range(4):
            assert abs(oracle.lagrange(x, j, x[i]) - (1.0 if i == j else 0.0)) < 1e-15
