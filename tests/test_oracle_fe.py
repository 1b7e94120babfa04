"""Pins of oracle/fe.py: closed forms and exact integration."""
import math

import numpy as np
import pytest
from numpy.polynomial import Polynomial

from oracle import fe


def test_gll_closed_forms():
    assert np.allclose(fe.gll_nodes(1), [0, 1], atol=0)
    assert np.allclose(fe.gll_nodes(2), [0, 0.5, 1], atol=1e-15)
    a = 0.5 * (1 - 1 / math.sqrt(5))
    assert np.allclose(fe.gll_nodes(3), [0, a, 1 - a, 1], atol=1e-15)
    b = 0.5 * (1 - math.sqrt(3.0 / 7.0))
    assert np.allclose(fe.gll_nodes(4), [0, b, 0.5, 1 - b, 1], atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gauss_exact_for_degree_2n_minus_1(n):
    x, w = fe.gauss(n)
    for p in range(2 * n):
        assert abs(np.sum(w * x ** p) - 1.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_lagrange_property_and_derivative(k):
    xi = fe.gll_nodes(k)
    assert np.allclose(fe.lagrange_values(xi, xi), np.eye(k + 1), atol=1e-14)
    # derivative against the exact derivative of the interpolating polynomial
    t = np.linspace(0, 1, 7)
    for a in range(k + 1):
        P = Polynomial.fromroots(np.delete(xi, a))
        P = P / P(xi[a])
        assert np.allclose(fe.lagrange_derivs(xi, t)[:, a], P.deriv()(t), atol=1e-11)


def _exact_1d(k):
    """1D mass and stiffness matrices on [0,1]: the Lagrange polynomials are
    built in monomial form and integrated with scipy's 12-point Gauss rule,
    which is exact for the degree-2k integrands."""
    from scipy.special import roots_legendre
    xi = fe.gll_nodes(k)
    basis = []
    for a in range(k + 1):
        P = Polynomial.fromroots(np.delete(xi, a))
        basis.append(P / P(xi[a]))
    t, w = roots_legendre(12)
    t, w = 0.5 * (t + 1), 0.5 * w
    V = np.array([b(t) for b in basis])
    D = np.array([b.deriv()(t) for b in basis])
    return (V * w) @ V.T, (D * w) @ D.T


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_element_matrix_closed_form(k):
    M, K = _exact_1d(k)
    # local index n = a + (k+1) b + (k+1)^2 c -> kron(z, kron(y, x))
    closed = np.kron(M, np.kron(M, K)) + np.kron(M, np.kron(K, M)) + np.kron(K, np.kron(M, M))
    A = fe.reference_laplace_matrix(k)
    assert np.abs(A - closed).max() < 1e-12 * np.abs(closed).max()
    # constants are in the kernel, A is symmetric positive semi-definite
    assert np.abs(A.sum(axis=1)).max() < 1e-13
    assert np.abs(A - A.T).max() < 1e-14
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > -1e-12 and np.sum(ev < 1e-10) == 1


@pytest.mark.parametrize("k", [1, 2, 4])
def test_mass_matrix_closed_form(k):
    M, _ = _exact_1d(k)
    assert np.abs(fe.reference_mass_matrix(k) - np.kron(M, np.kron(M, M))).max() < 1e-14
