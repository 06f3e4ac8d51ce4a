"""Oracle: geometric multigrid V-cycle with a Chebyshev-Jacobi smoother (test infrastructure).

Part of the CPU oracle (plain float64, never called by the product path).

Section 4.3: the matrix-free solver is preconditioned by geometric multigrid
with a polynomial (Chebyshev) variant of point-Jacobi as smoother; the
Chebyshev parameters come from an estimate of the largest eigenvalue by 10
CG / Lanczos iterations, the smoothing range is [0.08, 1.2] times that
estimate; transfers between levels are matrix-vector products.

Level hierarchy (the reading taken here; the paper uses h-multigrid at fixed p
on an octree, the workloads ask for p-coarsening followed by h-coarsening):

* p-levels on the fine mesh: p -> max(1, p // 2) -> ... -> 1, with the nodal
  interpolation of Q_pc into Q_pf as prolongation;
* h-levels at p = 1: each direction's n elements become ceil(n / 2) coarse
  elements made of every other vertex (a trailing odd element stays single);
  the prolongation evaluates the coarse trilinear function at each fine vertex
  placed at the reference coordinates -1, 0, +1 of its coarse element (for a
  single trailing element: -1, +1), which is the nodal interpolation on nested
  meshes and a fixed, mesh-independent transfer on perturbed ones;
* restriction = prolongation^T; coarse operators are rediscretised
  (alpha M_l + K_l on each level); a coarse element takes the tissue of its
  first fine child (lowest x, y, z);
* coarsening (p first, then h) goes on while a level has more than
  ``min_coarse_dofs`` nodes and can be coarsened further, so a p-level may be
  the coarsest one.

Chebyshev semi-iteration for A x = b with preconditioner D^{-1} on the
interval [a, b] of the spectrum of D^{-1} A (theta = (b+a)/2, delta = (b-a)/2,
sigma = theta/delta, rho_0 = 1/sigma):
  d_0 = D^{-1} r_0 / theta,  x_1 = x_0 + d_0
  rho_k = 1 / (2 sigma - rho_{k-1}),
  d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^{-1} r_k,  x_{k+1} = x_k + d_k.
The eigenvalue estimate runs 10 Jacobi-preconditioned CG iterations from a
fixed start vector and takes the largest eigenvalue of the Lanczos
tridiagonal matrix built from the CG coefficients.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import SlabSpace, assemble
from .quadrature import gll_rule, lagrange


def start_vector(n: int) -> np.ndarray:
    """Deterministic start vector of the eigenvalue estimate:
    v_i = ((i * 2654435761) mod 2^32) / 2^32 - 1/2 (Knuth's multiplicative hash)."""
    i = np.arange(n, dtype=np.uint64)
    h = (i * np.uint64(2654435761)) % np.uint64(2 ** 32)
    return h.astype(np.float64) / 2.0 ** 32 - 0.5


def lanczos_lambda_max(A, dinv, iters: int = 10) -> float:
    """Largest eigenvalue of D^{-1} A estimated from `iters` preconditioned CG steps."""
    n = A.shape[0]
    b = start_vector(n)
    x = np.zeros(n)
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = r @ z
    alphas, betas = [], []
    for _ in range(min(iters, n)):
        Ap = A @ p
        pAp = p @ Ap
        alpha = rz / pAp
        x += alpha * p
        r -= alpha * Ap
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
        if rz <= 0.0:
            break
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return float(np.linalg.eigvalsh(T).max())


def chebyshev(A, dinv, b, x0, degree: int, lo: float, hi: float):
    """`degree` steps of the Chebyshev semi-iteration (x0 = None means zero)."""
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x if x0 is not None else b.copy()
    d = dinv * r / theta
    x += d
    rho_old = 1.0 / sigma
    for _ in range(1, degree):
        r = b - A @ x
        rho = 1.0 / (2.0 * sigma - rho_old)
        d = rho * rho_old * d + (2.0 * rho / delta) * (dinv * r)
        x += d
        rho_old = rho
    return x


def p_prolongation(coarse: SlabSpace, fine: SlabSpace):
    """Nodal interpolation of Q_pc into Q_pf on the same mesh, as a sparse matrix."""
    xc, _ = gll_rule(coarse.p)
    xf, _ = gll_rule(fine.p)
    L = lagrange(xc, xf)  # [coarse node, fine point]
    nf, nc = fine.n, coarse.n
    seen = set()
    entries = {}
    for e in range(fine.nelem):
        df = fine.element_dofs(e)
        dc = coarse.element_dofs(e)
        for k in range(nf):
            for j in range(nf):
                for i in range(nf):
                    g = df[i + nf * (j + nf * k)]
                    if g in seen:
                        continue
                    seen.add(g)
                    for c in range(nc):
                        for b in range(nc):
                            for a in range(nc):
                                w = L[a, i] * L[b, j] * L[c, k]
                                if w != 0.0:
                                    entries[(g, dc[a + nc * (b + nc * c)])] = w
    r = np.array([k[0] for k in entries], dtype=np.int64)
    c = np.array([k[1] for k in entries], dtype=np.int64)
    v = np.array(list(entries.values()))
    return sp.csr_matrix((v, (r, c)), shape=(fine.ndofs, coarse.ndofs))


def _coarse_1d(nf: int):
    """Fine-vertex -> (coarse vertex indices, weights) along one direction."""
    nc = (nf + 1) // 2
    out = []
    for I in range(nf + 1):
        k = min(I // 2, nc - 1)
        span = 2 if 2 * k + 2 <= nf else 1
        t = I - 2 * k
        xi = -1.0 + 2.0 * t / span
        out.append(((k, k + 1), (0.5 * (1.0 - xi), 0.5 * (1.0 + xi))))
    return nc, out


def coarse_vertices(space: SlabSpace):
    """Vertices of the 2:1 coarsened mesh: every other fine vertex, plus the last."""
    V = space.V
    sel = [np.minimum(2 * np.arange((n + 1) // 2 + 1), n) for n in (space.nx, space.ny, space.nz)]
    return V[np.ix_(sel[2], sel[1], sel[0])], tuple((n + 1) // 2 for n in (space.nx, space.ny, space.nz))


def h_prolongation(coarse: SlabSpace, fine: SlabSpace):
    """Trilinear prolongation between 2:1 nested vertex lattices (p = 1)."""
    assert coarse.p == 1 and fine.p == 1
    ncx, mx = _coarse_1d(fine.nx)
    ncy, my = _coarse_1d(fine.ny)
    ncz, mz = _coarse_1d(fine.nz)
    assert (ncx, ncy, ncz) == (coarse.nx, coarse.ny, coarse.nz)
    rows, cols, vals = [], [], []
    NXc, NYc = ncx + 1, ncy + 1
    for K in range(fine.nz + 1):
        for J in range(fine.ny + 1):
            for I in range(fine.nx + 1):
                g = I + (fine.nx + 1) * (J + (fine.ny + 1) * K)
                (ix, wx), (iy, wy), (iz, wz) = mx[I], my[J], mz[K]
                for c in range(2):
                    for b in range(2):
                        for a in range(2):
                            w = wx[a] * wy[b] * wz[c]
                            if w != 0.0:
                                rows.append(g)
                                cols.append(ix[a] + NXc * (iy[b] + NYc * iz[c]))
                                vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.ndofs, coarse.ndofs))


def coarse_tissue(space: SlabSpace, tissue):
    """Per coarse element: the tissue of its first fine child."""
    ncx, ncy, ncz = ((n + 1) // 2 for n in (space.nx, space.ny, space.nz))
    idx = []
    for kz in range(ncz):
        for ky in range(ncy):
            for kx in range(ncx):
                idx.append(space.element_index(2 * kx, 2 * ky, 2 * kz))
    idx = np.array(idx)
    return tuple(np.asarray(t)[idx] for t in tissue)


class Hierarchy:
    """Levels, operators, Jacobi diagonals, transfers and smoother ranges."""

    def __init__(self, fine: SlabSpace, tissue, alpha: float, degree: int = 3,
                 coarse_degree: int = 10, min_coarse_dofs: int = 1000, lanczos_iters: int = 10,
                 range_lo: float = 0.08, range_hi: float = 1.2):
        self.degree, self.coarse_degree = degree, coarse_degree
        self.spaces = [fine]
        self.tissues = [tissue]
        self.P = []
        s, t = fine, tissue
        while s.p > 1 and s.ndofs > min_coarse_dofs:
            pc = max(1, s.p // 2)
            c = SlabSpace(s.V.reshape(-1, 3), s.nx, s.ny, s.nz, pc, s.quad)
            self.P.append(p_prolongation(c, s))
            self.spaces.append(c)
            self.tissues.append(t)
            s = c
        while s.ndofs > min_coarse_dofs and max(s.nx, s.ny, s.nz) > 1:
            Vc, (cx, cy, cz) = coarse_vertices(s)
            c = SlabSpace(Vc.reshape(-1, 3), cx, cy, cz, 1, s.quad)
            tc = coarse_tissue(s, t)
            self.P.append(h_prolongation(c, s))
            self.spaces.append(c)
            self.tissues.append(tc)
            s, t = c, tc
        self.A = [assemble(sp_, tis, alpha, 1.0) for sp_, tis in zip(self.spaces, self.tissues)]
        self.dinv = [1.0 / A.diagonal() for A in self.A]
        self.lam = [lanczos_lambda_max(A, d, lanczos_iters) for A, d in zip(self.A, self.dinv)]
        self.range = [(range_lo * lam, range_hi * lam) for lam in self.lam]

    @property
    def nlevels(self):
        return len(self.A)

    def vcycle(self, b, level: int = 0):
        A, dinv = self.A[level], self.dinv[level]
        lo, hi = self.range[level]
        if level == self.nlevels - 1:
            return chebyshev(A, dinv, b, None, self.coarse_degree, lo, hi)
        x = chebyshev(A, dinv, b, None, self.degree, lo, hi)
        r = b - A @ x
        xc = self.vcycle(self.P[level].T @ r, level + 1)
        x = x + self.P[level] @ xc
        return chebyshev(A, dinv, b, x, self.degree, lo, hi)

    def pcg(self, b, x0=None, rtol=1e-10, maxit=200):
        """Flexible PCG (Polak-Ribiere beta) preconditioned by one V-cycle."""
        A = self.A[0]
        x = np.zeros_like(b) if x0 is None else x0.copy()
        r = b - A @ x
        z = self.vcycle(r)
        p = z.copy()
        rz = r @ z
        tol = rtol * np.linalg.norm(b)
        it = 0
        while np.linalg.norm(r) > tol and it < maxit:
            Ap = A @ p
            alpha = rz / (p @ Ap)
            x += alpha * p
            r -= alpha * Ap
            z_old = z
            z = self.vcycle(r)
            rz_new = r @ z
            beta = (rz_new - r @ z_old) / rz
            rz = rz_new
            p = z + beta * p
            it += 1
        return x, it
