"""Pins of the oracle's SEM / SEM-NI operator (Sections 2-4).

Each check is fixed by the paper or by the mathematics, not by the oracle
itself:

* Q1 special case on the unit cube (SEM = FEM, SEM-NI = FEM with the
  trapezoidal rule): known Q1 element entries.
* K 1 = 0 (Neumann operator), symmetry, SEM-NI mass diagonal.
* 1^T M 1 = domain volume on a perturbed slab (LG always; LGL for p >= 2).
* Exact integration on affine meshes: u^T M v and u^T K v equal the closed-form
  integrals of polynomial fields (LG: u, v in Q_p; LGL: one factor of degree
  p-1), for an axis-aligned box and for a sheared parallelepiped.
* SEM-NI mass equals the row-sum lumping of the SEM mass on affine meshes
  (the ICI / lumped-ICI remark after Eq. algebraic_ionic).
* The printed Niederer DOF and cell counts.
* Assembled sparse operator (Algorithm 2) == element-by-element apply ==
  sampled rows.
* The conductivity tensor (Eq. diffusiontensor): eigenvalue sigma_l along the
  fibre (cos theta, sin theta, 0) and sigma_t across it, diagonal at theta = 0
  and pi/2; and through the assembled K, the energy of a linear field along
  and across the fibre is the volume times sigma_l and sigma_t.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import element as E
from oracle import mesh as Mh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _space(s, p, quad):
    return Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)


def test_q1_unit_cube_entries():
    s = W.slab(1, 1, 1, (1.0, 1.0, 1.0))
    X = s.element_vertices()[0]
    M, K = E.element_matrices(X, 1, "LG", np.eye(3))
    assert np.allclose(np.diag(K), 1 / 3, atol=1e-15)
    assert np.allclose(np.diag(M), 1 / 27, atol=1e-15)
    # Q1 FEM mass: 1/27 * (1/2)^(number of differing coordinates) for the 8 corners
    assert np.isclose(M[0, 7], 1 / 216, atol=1e-15)
    assert np.isclose(K[0, 7], -1 / 12, atol=1e-15)
    Mni, _ = E.element_matrices(X, 1, "LGL", np.eye(3))
    assert np.allclose(Mni, np.eye(8) / 8, atol=1e-15)


@pytest.mark.parametrize("quad", ["LG", "LGL"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_element_invariants(p, quad):
    s = W.slab(2, 1, 1, (2.0, 1.0, 1.3), perturb=0.15, seed=11)
    X = s.element_vertices()[1]
    D = E.diffusion_tensor(0.12, 0.03, 0.7)
    M, K = E.element_matrices(X, p, quad, D)
    assert np.abs(K @ np.ones(len(K))).max() < 1e-13 * np.abs(K).max()
    assert np.abs(K - K.T).max() < 1e-14 * np.abs(K).max()
    assert np.abs(M - M.T).max() < 1e-15 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 0
    off = M - np.diag(np.diag(M))
    if quad == "LGL":
        assert np.abs(off).max() == 0.0
    else:
        assert np.abs(off).max() > 1e-6


@pytest.mark.parametrize("quad,pmin", [("LG", 1), ("LGL", 2)])
def test_volume_on_perturbed_slab(quad, pmin):
    s = W.slab(3, 2, 2, (20.0, 7.0, 3.0), perturb=0.1, seed=3)
    for p in range(pmin, 5):
        sp_ = _space(s, p, quad)
        M = Mh.assemble(sp_, W.constant_tissue(s), 1.0, 0.0)
        one = np.ones(sp_.ndofs)
        assert abs(one @ (M @ one) - 20.0 * 7.0 * 3.0) < 1e-11 * 420


def test_lgl_p1_volume_not_exact_on_perturbed_mesh():
    """The trapezoidal rule (LGL, p = 1) cannot integrate the quadratic det J of a
    perturbed trilinear cell, so the volume is only approximate there."""
    s = W.slab(3, 2, 2, (20.0, 7.0, 3.0), perturb=0.1, seed=3)
    sp_ = _space(s, 1, "LGL")
    M = Mh.assemble(sp_, W.constant_tissue(s), 1.0, 0.0)
    one = np.ones(sp_.ndofs)
    assert abs(one @ (M @ one) - 420.0) > 1e-9


def _poly_integral_box(ca, cb, lengths):
    """Exact integral over [0,Lx]x[0,Ly]x[0,Lz] of the product of two separable
    polynomials given as lists of 1-D power-series coefficient arrays."""
    out = 1.0
    P = np.polynomial.polynomial
    for d in range(3):
        prod = P.polymul(ca[d], cb[d])
        anti = P.polyint(prod)
        out *= P.polyval(lengths[d], anti) - P.polyval(0.0, anti)
    return out


def _nodal(xyz, c):
    P = np.polynomial.polynomial
    return P.polyval(xyz[:, 0], c[0]) * P.polyval(xyz[:, 1], c[1]) * P.polyval(xyz[:, 2], c[2])


@pytest.mark.parametrize("quad", ["LG", "LGL"])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_exact_integration_affine_box(p, quad):
    """u^T K v = int grad u . D grad v and u^T M v = int u v for polynomial u, v."""
    rng = np.random.default_rng(7 + p)
    L = (2.0, 1.5, 1.0)
    s = W.slab(2, 2, 1, L)
    sp_ = _space(s, p, quad)
    theta = 0.6
    D = E.diffusion_tensor(0.12, 0.03, theta)
    tissue = W.constant_tissue(s, 0.12, 0.03, theta)
    M, K = Mh.assemble_mass_stiffness(sp_, tissue)
    xyz = sp_.dof_coordinates()
    du = p
    dv = p if quad == "LG" else p - 1
    cu = [rng.uniform(-1, 1, du + 1) for _ in range(3)]
    cv = [rng.uniform(-1, 1, dv + 1) for _ in range(3)]
    u = _nodal(xyz, cu)
    v = _nodal(xyz, cv)
    P = np.polynomial.polynomial
    exact_K = 0.0
    for a in range(3):
        for b in range(3):
            ga = [P.polyder(cu[d]) if d == a else cu[d] for d in range(3)]
            gb = [P.polyder(cv[d]) if d == b else cv[d] for d in range(3)]
            exact_K += D[a, b] * _poly_integral_box(ga, gb, L)
    assert abs(u @ (K @ v) - exact_K) < 1e-12 * (1 + abs(exact_K))
    if quad == "LG":
        exact_M = _poly_integral_box(cu, cv, L)
        assert abs(u @ (M @ v) - exact_M) < 1e-12 * (1 + abs(exact_M))


@pytest.mark.parametrize("quad", ["LG", "LGL"])
def test_exact_integration_sheared_affine(quad):
    """Sheared parallelepiped (constant, non-diagonal Jacobian): the exact
    integral comes from numpy's high-order Gauss-Legendre rule on the unit cube."""
    p = 3
    A = np.array([[2.0, 0.3, 0.1], [0.2, 1.5, -0.25], [0.0, 0.15, 1.0]])
    base = W.slab(2, 1, 2, (1.0, 1.0, 1.0))
    Vs = base.flat_vertices() @ A.T
    sp_ = Mh.SlabSpace(Vs, 2, 1, 2, p, quad)
    D = E.diffusion_tensor(0.12, 0.03, -0.4)
    tissue = W.constant_tissue(base, 0.12, 0.03, -0.4)
    M, K = Mh.assemble_mass_stiffness(sp_, tissue)
    xyz = sp_.dof_coordinates()

    # polynomials of total degree <= p (u) and <= p-1 (v) in x stay in Q_p of the affine cells
    def u_f(x):
        return x[:, 0] ** 3 - 2 * x[:, 0] * x[:, 1] * x[:, 2] + x[:, 1] ** 2 + 0.5

    def u_g(x):
        return np.stack([3 * x[:, 0] ** 2 - 2 * x[:, 1] * x[:, 2], -2 * x[:, 0] * x[:, 2] + 2 * x[:, 1],
                         -2 * x[:, 0] * x[:, 1]], axis=1)

    def v_f(x):
        return x[:, 0] * x[:, 2] - 3 * x[:, 1] ** 2 + x[:, 2]

    def v_g(x):
        return np.stack([x[:, 2], -6 * x[:, 1], x[:, 0] + 1.0], axis=1)

    t, w = np.polynomial.legendre.leggauss(10)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    g = np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3)
    wg = np.einsum("i,j,k->ijk", w, w, w).reshape(-1)
    x = g @ A.T
    detA = np.linalg.det(A)
    exact_K = detA * np.sum(wg * np.einsum("qa,ab,qb->q", u_g(x), D, v_g(x)))
    exact_M = detA * np.sum(wg * u_f(x) * v_f(x))
    u, v = u_f(xyz), v_f(xyz)
    assert abs(u @ (K @ v) - exact_K) < 1e-12 * (1 + abs(exact_K))
    if quad == "LG":
        assert abs(u @ (M @ v) - exact_M) < 1e-12 * (1 + abs(exact_M))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_semni_mass_is_lumped_sem_mass_on_affine_mesh(p):
    s = W.slab(3, 2, 1, (3.0, 2.0, 0.7))
    tissue = W.constant_tissue(s)
    Mlg = Mh.assemble(_space(s, p, "LG"), tissue, 1.0, 0.0)
    Mni = Mh.assemble(_space(s, p, "LGL"), tissue, 1.0, 0.0)
    lumped = np.asarray(Mlg.sum(axis=1)).ravel()
    assert np.allclose(Mni.diagonal(), lumped, rtol=1e-13, atol=1e-15)


def test_niederer_counts_golden():
    rows = np.loadtxt(os.path.join(GOLDEN, "niederer_counts.txt"), dtype=np.int64)
    for nx, ny, nz, p, npts, ncells in rows:
        s = Mh.SlabSpace(np.zeros(((nx + 1) * (ny + 1) * (nz + 1), 3)), nx, ny, nz, p, "LGL")
        assert s.ndofs == npts
        assert s.nelem == ncells


@pytest.mark.parametrize("quad", ["LG", "LGL"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_assembled_equals_element_by_element(p, quad):
    s = W.slab(3, 2, 2, (3.0, 2.0, 2.0), perturb=0.12, seed=5)
    sp_ = _space(s, p, quad)
    tissue = (np.linspace(0.1, 0.2, s.n_elements), np.linspace(0.02, 0.04, s.n_elements),
              W.transmural_fiber_angles(s))
    u = W.uniform_vector(sp_.ndofs)
    A = Mh.assemble(sp_, tissue, 2.5, 1.0)
    y1 = A @ u
    y2 = Mh.apply_element_by_element(sp_, tissue, u, 2.5, 1.0)
    idx = W.seeded_indices(sp_.ndofs, 25, seed=9)
    y3 = Mh.sampled_rows(sp_, tissue, u, idx, 2.5, 1.0)
    assert np.abs(y1 - y2).max() < 1e-13 * np.abs(y1).max()
    assert np.abs(y1[idx] - y3).max() < 1e-13 * np.abs(y1).max()
    dg = Mh.diagonal(sp_, tissue, 2.5, 1.0)
    assert np.allclose(dg, A.diagonal(), rtol=1e-14, atol=1e-14)


def test_global_stiffness_annihilates_constants():
    s = W.slab(4, 3, 2, (20.0, 7.0, 3.0), perturb=0.1)
    tissue = (np.full(s.n_elements, 0.12), np.full(s.n_elements, 0.03), W.transmural_fiber_angles(s))
    for quad in ("LG", "LGL"):
        sp_ = _space(s, 3, quad)
        K = Mh.assemble(sp_, tissue, 0.0, 1.0)
        assert np.abs(K @ np.ones(sp_.ndofs)).max() < 1e-14 * abs(K).max()


def test_diffusion_tensor_eigenstructure():
    """Eq. (diffusiontensor), transversely isotropic: the fibre direction
    f = (cos theta, sin theta, 0) is an eigenvector with eigenvalue sigma_l, and
    the plane normal to it (the sheet direction and the z axis) carries sigma_t.
    The axis-aligned angles fix the orientation convention."""
    sl, st = 0.12, 0.03
    assert np.allclose(E.diffusion_tensor(sl, st, 0.0), np.diag([sl, st, st]), atol=1e-17)
    assert np.allclose(E.diffusion_tensor(sl, st, np.pi / 2), np.diag([st, sl, st]), atol=1e-17)
    for theta in (0.3, -1.1, 2.5):
        D = E.diffusion_tensor(sl, st, theta)
        assert np.abs(D - D.T).max() == 0.0
        w, V = np.linalg.eigh(D)
        assert np.allclose(w, [st, st, sl], atol=1e-16)
        lead = V[:, 2] * np.sign(V[0, 2])
        ref = np.array([np.cos(theta), np.sin(theta), 0.0]) * np.sign(np.cos(theta))
        assert np.allclose(lead, ref, atol=1e-14)


@pytest.mark.parametrize("quad", ["LG", "LGL"])
def test_linear_field_energy_follows_the_fibre(quad):
    """For u = a . x on a box with a constant fibre angle, u^T K u is the volume
    times a^T D a: sigma_l along the fibre, sigma_t across it in the plane and
    along z.  This ties the per-element angle of the tissue arrays, through the
    assembled stiffness, to the physical fibre direction."""
    L = (2.0, 1.5, 1.0)
    vol = L[0] * L[1] * L[2]
    s = W.slab(2, 2, 1, L)
    sl, st, theta = 0.12, 0.03, 0.6
    for p in (1, 2):
        sp_ = _space(s, p, quad)
        _, K = Mh.assemble_mass_stiffness(sp_, W.constant_tissue(s, sl, st, theta))
        xyz = sp_.dof_coordinates()
        along = np.array([np.cos(theta), np.sin(theta), 0.0])
        across = np.array([-np.sin(theta), np.cos(theta), 0.0])
        for a, sigma in ((along, sl), (across, st), (np.array([0.0, 0.0, 1.0]), st)):
            u = xyz @ a
            assert abs(u @ (K @ u) - vol * sigma) < 1e-12 * vol * sigma, (p, a)
