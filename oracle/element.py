"""Oracle: dense element matrices of the SEM / SEM-NI operator (test infrastructure).

Part of the CPU oracle (plain float64, never called by the product path).

Section 2, Eq. (diffusiontensor): D = sigma_l f (x) f + sigma_t s (x) s +
sigma_n n (x) n.  Section 3: Q_p elements with the LGL nodal basis, LG
(SEM) or LGL (SEM-NI) quadrature with p+1 points per direction.
Section 4 / Algorithm 1: the cell loop computes the local mass matrix M_K
and stiffness matrix K_K of each cell and applies (alpha M_K + K_K) to the
local vector.

The oracle builds M_K and K_K as full dense (p+1)^3 x (p+1)^3 matrices by
summing over every quadrature point of the tensor rule, with the full 3-D
basis table -- no sum factorization:

  M_K[a, b] = sum_q  w_q |det J_q| phi_a(q) phi_b(q)
  K_K[a, b] = sum_q  w_q |det J_q| (J_q^{-T} grad phi_a(q)) . D (J_q^{-T} grad phi_b(q))

Geometry: each hexahedron is the trilinear image of [-1, 1]^3 through its 8
vertices (corner (a, b, c) in {0,1}^3 stored at index a + 2 b + 4 c).
"""
from __future__ import annotations

import functools

import numpy as np

from .quadrature import gll_rule, lagrange, lagrange_deriv, quadrature_rule

_CORNERS = np.array([[a, b, c] for c in range(2) for b in range(2) for a in range(2)], dtype=np.float64)
_SIGNS = 2.0 * _CORNERS - 1.0  # -1 or +1 per corner and direction


def trilinear_shape(xi):
    """N[v](xi) = prod_d (1 + s_vd xi_d) / 2 and dN[v, d] for points xi[..., 3]."""
    xi = np.asarray(xi, dtype=np.float64)
    f = 0.5 * (1.0 + _SIGNS[None, :, :] * xi.reshape(-1, 1, 3))  # [P, 8, 3]
    N = f.prod(axis=2)
    dN = np.empty(f.shape)
    for d in range(3):
        g = f.copy()
        g[:, :, d] = 0.5 * _SIGNS[None, :, d]
        dN[:, :, d] = g.prod(axis=2)
    return N, dN


def trilinear_map(X, xi):
    """Physical points x(xi) and Jacobians J[d, c] = dx_d / dxi_c of one hexahedron."""
    X = np.asarray(X, dtype=np.float64)
    N, dN = trilinear_shape(xi)
    x = N @ X
    J = np.einsum("pvc,vd->pdc", dN, X)
    return x, J


def diffusion_tensor(sigma_l: float, sigma_t: float, theta: float, sigma_n=None):
    """Eq. (diffusiontensor) with fibre f = (cos t, sin t, 0), sheetlet
    s = (-sin t, cos t, 0), sheet normal n = (0, 0, 1); sigma_n defaults to
    sigma_t (the transversely isotropic case)."""
    if sigma_n is None:
        sigma_n = sigma_t
    f = np.array([np.cos(theta), np.sin(theta), 0.0])
    s = np.array([-np.sin(theta), np.cos(theta), 0.0])
    nn = np.array([0.0, 0.0, 1.0])
    return sigma_l * np.outer(f, f) + sigma_t * np.outer(s, s) + sigma_n * np.outer(nn, nn)


def tensor_points(x1d):
    """3-D tensor points, index q = qx + n qy + n^2 qz (x fastest)."""
    n = len(x1d)
    pts = np.empty((n ** 3, 3))
    q = 0
    for qz in range(n):
        for qy in range(n):
            for qx in range(n):
                pts[q] = (x1d[qx], x1d[qy], x1d[qz])
                q += 1
    return pts


@functools.lru_cache(maxsize=None)
def basis_tables(p: int, quad: str):
    """phi[a, q], dphi[a, q, 3] of the (p+1)^3 nodal basis at the quadrature
    points, plus tensor weights w[q].  Basis index a = i + n j + n^2 k."""
    n = p + 1
    xg, _ = gll_rule(p)
    xq, wq = quadrature_rule(p, quad)
    L = lagrange(xg, xq)
    dL = lagrange_deriv(xg, xq)
    phi = np.einsum("iq,jr,ks->kjisrq", L, L, L).reshape(n ** 3, n ** 3)
    dphi = np.empty((n ** 3, n ** 3, 3))
    dphi[:, :, 0] = np.einsum("iq,jr,ks->kjisrq", dL, L, L).reshape(n ** 3, n ** 3)
    dphi[:, :, 1] = np.einsum("iq,jr,ks->kjisrq", L, dL, L).reshape(n ** 3, n ** 3)
    dphi[:, :, 2] = np.einsum("iq,jr,ks->kjisrq", L, L, dL).reshape(n ** 3, n ** 3)
    w = np.einsum("q,r,s->srq", wq, wq, wq).reshape(-1)
    return phi, dphi, w, tensor_points(xq)


def element_geometry(X, p: int, quad: str):
    """Quadrature weights times |det J| and J^{-T} at every quadrature point."""
    _, _, w, pts = basis_tables(p, quad)
    _, J = trilinear_map(X, pts)
    det = np.linalg.det(J)
    if np.any(det <= 0.0):
        raise ValueError("non-positive Jacobian determinant in element")
    JinvT = np.linalg.inv(J).transpose(0, 2, 1)
    return w * det, JinvT


def element_matrices(X, p: int, quad: str, D):
    """Dense local mass and stiffness matrices (M_K, K_K) of one hexahedron."""
    phi, dphi, w, pts = basis_tables(p, quad)
    _, J = trilinear_map(X, pts)
    det = np.linalg.det(J)
    if np.any(det <= 0.0):
        raise ValueError("non-positive Jacobian determinant in element")
    JinvT = np.linalg.inv(J).transpose(0, 2, 1)
    W = w * det
    grad = np.einsum("qcd,aqd->aqc", JinvT, dphi)  # physical gradients [a, q, 3]
    return _mass_stiffness(W, phi, grad, D, phi, grad)


def _mass_stiffness(W, phi_rows, grad_rows, D, phi, grad):
    """M[a, b] = sum_q W_q phi_a phi_b and K[a, b] = sum_q W_q grad_a . D grad_b,
    each written as one matrix product over the flattened (q, component) index."""
    D = np.asarray(D, dtype=np.float64)
    M = (phi_rows * W[None, :]) @ phi.T
    DG = np.einsum("aqc,cd->aqd", grad_rows, D) * W[None, :, None]
    na = grad_rows.shape[0]
    K = DG.reshape(na, -1) @ grad.reshape(grad.shape[0], -1).T
    return M, K


def element_matrix_rows(X, p: int, quad: str, D, rows):
    """Rows ``rows`` of M_K and K_K only (for sampled outputs of big meshes)."""
    phi, dphi, w, pts = basis_tables(p, quad)
    _, J = trilinear_map(X, pts)
    det = np.linalg.det(J)
    JinvT = np.linalg.inv(J).transpose(0, 2, 1)
    W = w * det
    grad = np.einsum("qcd,aqd->aqc", JinvT, dphi)
    rows = np.asarray(rows)
    return _mass_stiffness(W, phi[rows], grad[rows], D, phi, grad)
