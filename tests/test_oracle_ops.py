"""Pins for the oracle's 1D operators (Sec. 2.2, Eq. dgsem and the definitions of
Dhat and lhat after it; Nonlinear Stability for the split operator).

Every check here compares against something the oracle does not compute itself:
closed-form LGL nodes/weights, exact integrals and derivatives of monomials,
the summation-by-parts identity, and numpy's Legendre evaluation.
"""
import math

import numpy as np
import pytest

import oracle as O


def test_lgl_closed_forms():
    # N = 2: nodes {-1, 0, 1}, weights {1/3, 4/3, 1/3}
    x, w, *_ = O.ops(2)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-15)
    # N = 3: +-1, +-1/sqrt(5); weights 1/6, 5/6
    x, w, *_ = O.ops(3)
    s = 1 / math.sqrt(5)
    np.testing.assert_allclose(x, [-1, -s, s, 1], rtol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-15)
    # N = 4: 0, +-sqrt(3/7); weights 1/10, 49/90, 32/45
    x, w, *_ = O.ops(4)
    s = math.sqrt(3 / 7)
    np.testing.assert_allclose(x, [-1, -s, 0, s, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=1e-14)


@pytest.mark.parametrize("N", range(1, 13))
def test_lgl_quadrature_exactness(N):
    """Sum of weights is 2, quadrature exact up to degree 2N-1, inexact at 2N."""
    x, w, *_ = O.ops(N)
    assert abs(w.sum() - 2) < 1e-14
    for k in range(0, 2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13, k
    if N >= 1:
        k = 2 * N
        assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-10


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9])
def test_derivative_matrix_exact_on_polynomials(N):
    x, w, D, *_ = O.ops(N)
    for m in range(0, N + 1):
        dm = m * x ** (m - 1) if m > 0 else np.zeros_like(x)
        np.testing.assert_allclose(D @ x ** m, dm, atol=1e-11 * max(1, m * N * N))
    # degree N+1 is not differentiated exactly
    assert np.abs(D @ x ** (N + 1) - (N + 1) * x ** N).max() > 1e-6


@pytest.mark.parametrize("N", [1, 2, 3, 4, 7, 10])
def test_sbp_and_weak_and_split_operators(N):
    """W D + D^T W = diag(-1, 0, ..., 0, 1) (summation by parts);
    Dhat = D - e_N e_N^T / w_N + e_0 e_0^T / w_0 (the weak operator equals the
    strong one plus the two surface corrections, which is what makes the weight
    ratio of Dhat read as w_a / w_i); diag(Dsplit) = 0 on LGL."""
    x, w, D, Dh, Ds, _ = O.ops(N)
    W = np.diag(w)
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1, 1
    np.testing.assert_allclose(W @ D + D.T @ W, B, atol=1e-12 * N * N)
    C = D.copy()
    C[N, N] -= 1 / w[N]
    C[0, 0] += 1 / w[0]
    np.testing.assert_allclose(Dh, C, atol=1e-12 * N * N)
    np.testing.assert_allclose(np.diag(Ds), 0, atol=1e-12 * N * N)
    # split operator applied to a symmetric two-point function of a constant
    # reproduces the weak operator on that constant
    np.testing.assert_allclose(Ds.sum(axis=1), Dh.sum(axis=1), atol=1e-12 * N * N)


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_inverse_vandermonde_against_numpy_legendre(N):
    """Vinv maps nodal values of the orthonormal Legendre polynomial
    sqrt((2m+1)/2) P_m (evaluated by numpy) to the unit vector e_m."""
    x, _, _, _, _, Vinv = O.ops(N)
    for m in range(N + 1):
        c = np.zeros(m + 1)
        c[m] = 1.0
        vals = math.sqrt((2 * m + 1) / 2) * np.polynomial.legendre.legval(x, c)
        e = np.zeros(N + 1)
        e[m] = 1
        np.testing.assert_allclose(Vinv @ vals, e, atol=1e-12)


def test_quad_ops_agree_with_double():
    for N in (3, 7):
        d = O.ops(N)
        q = O.ops(N, quad=True)
        for a, b in zip(d, q):
            np.testing.assert_allclose(a, b, atol=1e-13 * N * N)
