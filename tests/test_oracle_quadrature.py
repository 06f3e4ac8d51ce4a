"""Pins of the oracle's 1-D rules and Lagrange basis (Section 3).

Textbook node/weight values, the exactness degrees the paper states
(LG with p+1 points exact to 2p+1, LGL with p+1 points exact to 2p-1), and
interpolation identities of the nodal basis."""
import math

import numpy as np
import pytest

from oracle import quadrature as Q


def test_gll_textbook_values():
    x, w = Q.gll_rule(2)
    assert np.allclose(x, [-1, 0, 1], atol=1e-15)
    assert np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = Q.gll_rule(3)
    a = 1 / math.sqrt(5)
    assert np.allclose(x, [-1, -a, a, 1], atol=1e-15)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    x, w = Q.gll_rule(4)
    b = math.sqrt(3 / 7)
    assert np.allclose(x, [-1, -b, 0, b, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


def test_gauss_textbook_values():
    x, w = Q.gauss_rule(2)
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1, 1], atol=1e-15)
    x, w = Q.gauss_rule(3)
    c = math.sqrt(3 / 5)
    assert np.allclose(x, [-c, 0, c], atol=1e-15)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


def _mono_exact(k):
    return 0.0 if k % 2 else 2.0 / (k + 1)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_lg_exactness_degree(p):
    """LG with p+1 points integrates x^k exactly for k <= 2p+1 and not k = 2p+2."""
    x, w = Q.gauss_rule(p + 1)
    for k in range(2 * p + 2):
        assert abs(w @ x ** k - _mono_exact(k)) < 1e-14
    assert abs(w @ x ** (2 * p + 2) - _mono_exact(2 * p + 2)) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_lgl_exactness_degree(p):
    """LGL with p+1 points integrates x^k exactly for k <= 2p-1 and not k = 2p."""
    x, w = Q.gll_rule(p)
    for k in range(2 * p):
        assert abs(w @ x ** k - _mono_exact(k)) < 1e-14
    assert abs(w @ x ** (2 * p) - _mono_exact(2 * p)) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_lgl_nodes_are_roots_of_legendre_derivative(p):
    """Interior LGL nodes agree with numpy's Legendre-series roots of P_p'."""
    x, _ = Q.gll_rule(p)
    c = np.zeros(p + 1)
    c[p] = 1.0
    r = np.sort(np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c)))
    assert np.allclose(x[1:-1], r, atol=1e-13)
    xg, wg = np.polynomial.legendre.leggauss(p + 1)
    xq, wq = Q.gauss_rule(p + 1)
    assert np.allclose(xq, xg, atol=1e-14) and np.allclose(wq, wg, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_lagrange_basis_identities(p):
    xg, _ = Q.gll_rule(p)
    L = Q.lagrange(xg, xg)
    assert np.allclose(L, np.eye(p + 1), atol=1e-14)
    t = np.linspace(-1, 1, 17)
    L = Q.lagrange(xg, t)
    dL = Q.lagrange_deriv(xg, t)
    for k in range(p + 1):
        # reproduction of x^k and of its derivative
        assert np.allclose(xg ** k @ L, t ** k, atol=1e-13)
        assert np.allclose(xg ** k @ dL, k * t ** max(k - 1, 0) if k else 0 * t, atol=1e-12)


def test_lagrange_derivative_matches_numpy_polyfit():
    """l_i' from the product formula equals the derivative of the interpolating
    polynomial obtained by numpy's polynomial fit through the nodes."""
    xg, _ = Q.gll_rule(5)
    t = np.linspace(-0.9, 0.9, 7)
    dL = Q.lagrange_deriv(xg, t)
    for i in range(6):
        e = np.zeros(6)
        e[i] = 1.0
        c = np.polynomial.polynomial.polyfit(xg, e, 5)
        d = np.polynomial.polynomial.polyval(t, np.polynomial.polynomial.polyder(c))
        assert np.allclose(dL[i], d, atol=1e-10)
