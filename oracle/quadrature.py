"""Oracle: 1-D quadrature rules and the nodal Lagrange basis (test infrastructure).

This file is part of the CPU oracle, a slow, plain float64 restatement of the
paper's method that the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` compare the CUDA path against.  Nothing in the
product path imports it.

Section 3 (space discretization): the nodal basis of Q_p is the Lagrange
basis on the p+1 Legendre--Gauss--Lobatto (LGL) nodes of [-1, 1]; SEM
integrates with the (p+1)-point Legendre--Gauss (LG) rule (exact to degree
2p+1), SEM-NI with the (p+1)-point LGL rule (exact to degree 2p-1), whose
nodes coincide with the basis nodes.

Everything is written from the textbook definitions:

* Legendre polynomials by the three-term recurrence
  (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}.
* LGL nodes: x = -1, +1 and the p-1 roots of P_p'; weights
  2 / (p (p+1) P_p(x)^2).
* LG nodes: the n roots of P_n; weights 2 / ((1 - x^2) P_n'(x)^2).
* Lagrange basis and its derivative by the product formula (no barycentric
  weights, no differentiation-matrix shortcut).
"""
from __future__ import annotations

import numpy as np


def legendre(n: int, x):
    """P_n(x), P_n'(x) by the three-term recurrence (x may be an array)."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    d0 = np.zeros_like(x)
    d1 = np.ones_like(x)
    for k in range(1, n):
        p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        # derivative of the same recurrence
        d2 = ((2 * k + 1) * (p1 + x * d1) - k * d0) / (k + 1)
        p0, p1 = p1, p2
        d0, d1 = d1, d2
    return p1, d1


def _newton(f, x0, iters=100):
    x = np.array(x0, dtype=np.float64)
    for _ in range(iters):
        fx, dfx = f(x)
        dx = fx / dfx
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    return x


def gauss_rule(n: int):
    """n-point Legendre--Gauss rule on [-1, 1]: (nodes ascending, weights)."""
    if n < 1:
        raise ValueError("n >= 1")
    k = np.arange(n)
    x0 = -np.cos(np.pi * (k + 0.75) / (n + 0.5))
    x = _newton(lambda t: legendre(n, t), x0)
    x = np.sort(x)
    _, dp = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def gll_rule(p: int):
    """(p+1)-point Legendre--Gauss--Lobatto rule on [-1, 1]: (nodes ascending, weights)."""
    if p < 1:
        raise ValueError("p >= 1")
    if p == 1:
        return np.array([-1.0, 1.0]), np.array([1.0, 1.0])

    def f(t):
        # root finding on P_p'; its derivative from Legendre's equation
        # (1 - t^2) P'' = 2 t P' - p (p+1) P
        pp, dp = legendre(p, t)
        d2 = (2.0 * t * dp - p * (p + 1) * pp) / (1.0 - t * t)
        return dp, d2

    k = np.arange(1, p)
    x0 = -np.cos(np.pi * k / p)
    inner = _newton(f, x0)
    x = np.concatenate(([-1.0], np.sort(inner), [1.0]))
    pp, _ = legendre(p, x)
    w = 2.0 / (p * (p + 1) * pp * pp)
    return x, w


def lagrange(nodes, x):
    """Values L[i, q] = l_i(x_q) of the Lagrange basis on ``nodes`` (product formula)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    L = np.ones((n, x.size))
    for i in range(n):
        for m in range(n):
            if m != i:
                L[i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
    return L


def lagrange_deriv(nodes, x):
    """Derivatives dL[i, q] = l_i'(x_q) by differentiating the product formula:
    l_i'(x) = sum_{m != i} 1/(x_i - x_m) prod_{l != i, m} (x - x_l)/(x_i - x_l)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    dL = np.zeros((n, x.size))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(x.size, 1.0 / (nodes[i] - nodes[m]))
            for l in range(n):
                if l != i and l != m:
                    term *= (x - nodes[l]) / (nodes[i] - nodes[l])
            dL[i] += term
    return dL


def quadrature_rule(p: int, quad: str):
    """The (p+1)-point rule of the method: 'LG' for SEM, 'LGL' for SEM-NI (Section 3)."""
    if quad == "LG":
        return gauss_rule(p + 1)
    if quad == "LGL":
        return gll_rule(p)
    raise ValueError(f"unknown quadrature {quad!r}")
