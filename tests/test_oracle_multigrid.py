"""Pins of the oracle's geometric multigrid (Section 4.3).

* Prolongations: nodal interpolation reproduces Q_pc fields on Q_pf nodes
  exactly, and the 2:1 vertex transfer reproduces trilinear fields on a nested
  (unperturbed) mesh, for even and odd element counts.
* Chebyshev smoother: its error-propagation operator acts on each generalized
  eigenvector of (A, D) as the closed-form Chebyshev polynomial
  T_k((theta - lambda) / delta) / T_k(theta / delta).
* Lanczos estimate: below the true largest eigenvalue of D^{-1} A and within
  a few percent of it.
* V-cycle: a symmetric operator; PCG with it reaches the direct solution in
  few iterations.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import workloads as W
from oracle import mesh as Mh
from oracle import multigrid as MG


def _space(s, p, quad="LGL"):
    return Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)


@pytest.mark.parametrize("pf,pc", [(2, 1), (4, 2), (6, 3), (3, 1), (5, 2)])
def test_p_prolongation_reproduces_coarse_polynomials(pf, pc):
    s = W.slab(3, 2, 2, (3.0, 2.0, 1.0))
    f, c = _space(s, pf), _space(s, pc)
    P = MG.p_prolongation(c, f)
    rng = np.random.default_rng(1)
    cx, cy, cz = (rng.uniform(-1, 1, pc + 1) for _ in range(3))
    P1 = np.polynomial.polynomial.polyval

    def fn(xyz):
        return P1(xyz[:, 0], cx) * P1(xyz[:, 1], cy) * P1(xyz[:, 2], cz)

    assert np.abs(P @ fn(c.dof_coordinates()) - fn(f.dof_coordinates())).max() < 1e-12


@pytest.mark.parametrize("dims", [(4, 2, 2), (5, 3, 1), (7, 4, 3)])
def test_h_prolongation_reproduces_trilinear_fields(dims):
    s = W.slab(*dims, (2.0, 1.5, 1.0))
    f = _space(s, 1)
    Vc, (cx, cy, cz) = MG.coarse_vertices(f)
    c = Mh.SlabSpace(Vc.reshape(-1, 3), cx, cy, cz, 1, "LGL")
    P = MG.h_prolongation(c, f)

    def fn(xyz):
        return (1 + 2 * xyz[:, 0]) * (3 - xyz[:, 1]) * (0.5 + xyz[:, 2])

    assert np.abs(P @ fn(c.dof_coordinates()) - fn(f.dof_coordinates())).max() < 1e-13
    # each fine vertex's weights sum to one
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0)


@pytest.mark.parametrize("degree", [2, 3, 5])
def test_chebyshev_error_polynomial(degree):
    s = W.slab(3, 2, 1, (3.0, 2.0, 1.0), perturb=0.1)
    sp_ = _space(s, 2)
    A = Mh.assemble(sp_, W.constant_tissue(s), 30.0, 1.0).toarray()
    d = np.diag(A)
    dinv = 1.0 / d
    lam, V = sla.eigh(A, np.diag(d))
    lo, hi = 0.08 * lam.max(), 1.2 * lam.max()
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    n = A.shape[0]
    # error propagation E = I - S A, S the smoother's linear map (zero start)
    S = np.stack([MG.chebyshev(A, dinv, np.eye(n)[:, j], None, degree, lo, hi) for j in range(n)], axis=1)
    E = np.eye(n) - S @ A
    T = np.polynomial.chebyshev.Chebyshev.basis(degree)
    expected = T((theta - lam) / delta) / T(theta / delta)
    got = np.einsum("ij,ij->j", V, E @ V) / np.einsum("ij,ij->j", V, V)
    assert np.abs(got - expected).max() < 1e-10
    inside = lam >= lo
    assert np.abs(got[inside]).max() <= 1.0 / abs(T(theta / delta)) + 1e-12


def test_lanczos_estimate_bounds_lambda_max():
    s = W.slab(4, 3, 2, (4.0, 3.0, 2.0), perturb=0.1)
    sp_ = _space(s, 2, "LG")
    A = Mh.assemble(sp_, W.constant_tissue(s, 0.12, 0.03, 0.5), 30.0, 1.0)
    d = A.diagonal()
    est = MG.lanczos_lambda_max(A, 1.0 / d, 10)
    true = float(sla.eigh(A.toarray(), np.diag(d), eigvals_only=True).max())
    assert est <= true * (1 + 1e-12)
    assert est > 0.9 * true


@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_vcycle_symmetric_and_pcg_converges(quad):
    s = W.slab(6, 4, 3, (20.0, 7.0, 3.0), perturb=0.1)
    tissue = (np.full(s.n_elements, 0.12), np.full(s.n_elements, 0.03), W.transmural_fiber_angles(s))
    sp_ = _space(s, 4, quad)
    H = MG.Hierarchy(sp_, tissue, 30.0, degree=3, coarse_degree=10, min_coarse_dofs=30)
    assert H.nlevels >= 4 and H.spaces[-1].p == 1
    y = W.uniform_vector(sp_.ndofs, seed=3)
    z = W.uniform_vector(sp_.ndofs, seed=4)
    a, b = z @ H.vcycle(y), y @ H.vcycle(z)
    assert abs(a - b) < 1e-11 * abs(a)
    x, it = H.pcg(y, rtol=1e-12)
    xref = spla.spsolve(H.A[0].tocsc(), y)
    assert np.linalg.norm(x - xref) < 1e-10 * np.linalg.norm(xref)
    assert it <= 15, it


@pytest.mark.parametrize("min_coarse,ps", [(1000, [4, 2]), (500, [4, 2, 1]), (100, [4, 2, 1, 1])])
def test_coarsening_stops_at_first_small_level(min_coarse, ps):
    """p-levels of the 6 x 4 x 3 slab at p = 4 have 5525, 819 and 140 nodes; coarsening
    (p first, then h) stops at the first level with at most min_coarse_dofs nodes."""
    s = W.slab(6, 4, 3, (20.0, 7.0, 3.0), perturb=0.1)
    tissue = (np.full(s.n_elements, 0.12), np.full(s.n_elements, 0.03), W.transmural_fiber_angles(s))
    H = MG.Hierarchy(_space(s, 4, "LGL"), tissue, 30.0, degree=3, coarse_degree=10,
                     min_coarse_dofs=min_coarse)
    assert [sp_.p for sp_ in H.spaces] == ps
    assert [sp_.ndofs for sp_ in H.spaces][:3] == [5525, 819, 140][:len(ps)]
    assert H.spaces[-1].ndofs <= min_coarse
    assert all(sp_.ndofs > min_coarse for sp_ in H.spaces[:-1])
