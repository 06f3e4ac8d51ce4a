"""Oracle: global DOF numbering, assembly and matrix-based operator (test infrastructure).

Part of the CPU oracle (plain float64, never called by the product path).

Section 3: V_{h,p} is the space of globally continuous piecewise Q_p
functions on a conforming hexahedral mesh.  On a structured slab of
nx x ny x nz hexahedra the LGL nodes of neighbouring elements coincide on
shared faces, so the global nodes form a (p nx + 1) x (p ny + 1) x
(p nz + 1) lattice, numbered here with x fastest.

Section 4, Algorithm 2 (matrix-based workflow): the local matrices
alpha M_K + K_K are "compressed" (assembled) into one global sparse matrix
A, and y = A u is a sparse matrix-vector product.  For meshes too large to
assemble, ``apply_element_by_element`` and ``sampled_rows`` compute the same
y = A u from dense local matrices, one element at a time.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .element import (diffusion_tensor, element_geometry, element_matrices, element_matrix_rows,
                      trilinear_map, tensor_points)
from .quadrature import gll_rule


class SlabSpace:
    """Q_p space on a structured slab given by its vertex lattice."""

    def __init__(self, vertices, nx: int, ny: int, nz: int, p: int, quad: str):
        self.nx, self.ny, self.nz, self.p, self.quad = nx, ny, nz, p, quad
        self.n = p + 1
        self.V = np.asarray(vertices, dtype=np.float64).reshape(nz + 1, ny + 1, nx + 1, 3)
        self.NX, self.NY, self.NZ = p * nx + 1, p * ny + 1, p * nz + 1
        self.ndofs = self.NX * self.NY * self.NZ
        self.nelem = nx * ny * nz

    # --- numbering -----------------------------------------------------
    def element_index(self, ex, ey, ez):
        return ex + self.nx * (ey + self.ny * ez)

    def element_ijk(self, e):
        ex = e % self.nx
        ey = (e // self.nx) % self.ny
        ez = e // (self.nx * self.ny)
        return ex, ey, ez

    def element_vertices(self, e):
        ex, ey, ez = self.element_ijk(e)
        X = np.empty((8, 3))
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    X[a + 2 * b + 4 * c] = self.V[ez + c, ey + b, ex + a]
        return X

    def element_dofs(self, e):
        """Global indices of the local nodes a = i + n j + n^2 k of element e."""
        ex, ey, ez = self.element_ijk(e)
        n, p = self.n, self.p
        k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        g = (ex * p + i) + self.NX * ((ey * p + j) + self.NY * (ez * p + k))
        return g.reshape(-1)

    def elements_of_dof(self, g):
        """Elements whose closure holds global node g."""
        I = g % self.NX
        J = (g // self.NX) % self.NY
        K = g // (self.NX * self.NY)
        p = self.p

        def cand(I, nel):
            c = {I // p}
            if I % p == 0:
                c.add(I // p - 1)
            return [x for x in c if 0 <= x < nel]

        out = []
        for ez in cand(K, self.nz):
            for ey in cand(J, self.ny):
                for ex in cand(I, self.nx):
                    out.append(self.element_index(ex, ey, ez))
        return sorted(out)

    # --- geometry ------------------------------------------------------
    def dof_coordinates(self):
        """Physical coordinates [ndofs, 3] of the global nodes (trilinear image of the
        LGL tensor points of each element)."""
        xg, _ = gll_rule(self.p)
        pts = tensor_points(xg)
        xyz = np.empty((self.ndofs, 3))
        for e in range(self.nelem):
            x, _ = trilinear_map(self.element_vertices(e), pts)
            xyz[self.element_dofs(e)] = x
        return xyz

    def volume_weights(self, e):
        W, _ = element_geometry(self.element_vertices(e), self.p, self.quad)
        return W


def _tensor(tissue, e):
    sl, st, th = tissue
    return diffusion_tensor(sl[e], st[e], th[e])


def assemble(space: SlabSpace, tissue, alpha: float = 1.0, beta: float = 1.0):
    """Global sparse A = alpha M + beta K (CSR), Algorithm 2's assembly phase."""
    rows, cols, vals = [], [], []
    for e in range(space.nelem):
        M, K = element_matrices(space.element_vertices(e), space.p, space.quad, _tensor(tissue, e))
        A = alpha * M + beta * K
        d = space.element_dofs(e)
        rows.append(np.repeat(d, d.size))
        cols.append(np.tile(d, d.size))
        vals.append(A.reshape(-1))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(space.ndofs, space.ndofs))
    return A.tocsr()


def assemble_mass_stiffness(space: SlabSpace, tissue):
    """(M, K) as separate global CSR matrices."""
    return assemble(space, tissue, 1.0, 0.0), assemble(space, tissue, 0.0, 1.0)


def apply_element_by_element(space: SlabSpace, tissue, u, alpha: float = 1.0, beta: float = 1.0,
                             elements=None):
    """y = (alpha M + beta K) u from dense local matrices, element by element
    (Algorithm 1's cell loop without sum factorization).  With ``elements``
    only those elements contribute (a bounded sample)."""
    u = np.asarray(u, dtype=np.float64)
    y = np.zeros(space.ndofs)
    it = range(space.nelem) if elements is None else elements
    for e in it:
        M, K = element_matrices(space.element_vertices(e), space.p, space.quad, _tensor(tissue, e))
        d = space.element_dofs(e)
        y[d] += (alpha * M + beta * K) @ u[d]
    return y


def sampled_rows(space: SlabSpace, tissue, u, dofs, alpha: float = 1.0, beta: float = 1.0):
    """y_g = ((alpha M + beta K) u)_g for the global nodes g in ``dofs`` only."""
    u = np.asarray(u, dtype=np.float64)
    out = np.empty(len(dofs))
    for t, g in enumerate(dofs):
        acc = 0.0
        for e in space.elements_of_dof(int(g)):
            d = space.element_dofs(e)
            a = int(np.nonzero(d == g)[0][0])
            M, K = element_matrix_rows(space.element_vertices(e), space.p, space.quad,
                                       _tensor(tissue, e), [a])
            acc += float((alpha * M[0] + beta * K[0]) @ u[d])
        out[t] = acc
    return out


def diagonal(space: SlabSpace, tissue, alpha: float = 1.0, beta: float = 1.0):
    """diag(alpha M + beta K), summed over elements."""
    dg = np.zeros(space.ndofs)
    for e in range(space.nelem):
        M, K = element_matrices(space.element_vertices(e), space.p, space.quad, _tensor(tissue, e))
        dg[space.element_dofs(e)] += alpha * np.diag(M) + beta * np.diag(K)
    return dg
