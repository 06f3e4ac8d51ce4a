"""Convergence pins of the oracle (Section 3, Eq. sem_error; Appendix).

* Space: a manufactured reaction-diffusion problem with homogeneous Neumann
  data, -div(D grad u) + c u = f on the unit cube with
  u = cos(pi x) cos(pi y) cos(pi z) (the Appendix's test solutions do not
  satisfy the paper's Neumann condition; this one does).  The L2 error of the
  SEM and SEM-NI solutions decays with order p + 1 under h-refinement.
* Time: the partitioned scheme (BDF1 start, then BDF2 with the extrapolated
  u*) on u = (2 + sin(pi t)) q(x), q(x) = x^2 (3L - 2x), which Q_3 represents
  exactly (the Appendix's device of a solution exact in space), with a linear
  reaction I_ion = beta u: the error at the final time is O(dt^2).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import element as E
from oracle import mesh as Mh
from oracle import monodomain as MD
from oracle import quadrature as Q


def _l2_error(space, uh, exact):
    """||u_h - u||_L2 with a 7-point-per-direction Gauss rule per element."""
    t, w = np.polynomial.legendre.leggauss(7)
    pts = E.tensor_points(t)
    wq = np.einsum("q,r,s->srq", w, w, w).reshape(-1)
    xg, _ = Q.gll_rule(space.p)
    L = Q.lagrange(xg, t)
    phi = np.einsum("iq,jr,ks->kjisrq", L, L, L).reshape((space.p + 1) ** 3, -1)
    err2 = 0.0
    for e in range(space.nelem):
        X = space.element_vertices(e)
        x, J = E.trilinear_map(X, pts)
        det = np.linalg.det(J)
        val = uh[space.element_dofs(e)] @ phi
        err2 += np.sum(wq * det * (val - exact(x)) ** 2)
    return np.sqrt(err2)


@pytest.mark.parametrize("quad", ["LG", "LGL"])
@pytest.mark.parametrize("p,levels", [(1, (4, 8)), (2, (2, 4)), (3, (2, 4)), (4, (1, 2))])
def test_spatial_order_p_plus_one(p, levels, quad):
    sl, st, c = 0.12, 0.03, 1.0

    def exact(x):
        return np.cos(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]) * np.cos(np.pi * x[:, 2])

    errs = []
    for N in levels:
        s = W.slab(N, N, N, (1.0, 1.0, 1.0))
        sp_ = Mh.SlabSpace(s.flat_vertices(), N, N, N, p, quad)
        tissue = W.constant_tissue(s, sl, st, 0.0)
        M, K = Mh.assemble_mass_stiffness(sp_, tissue)
        xyz = sp_.dof_coordinates()
        f = (np.pi ** 2 * (sl + 2 * st) + c) * exact(xyz)
        uh = spla.spsolve((K + c * M).tocsc(), M @ f)
        errs.append(_l2_error(sp_, uh, exact))
    order = np.log(errs[0] / errs[1]) / np.log(levels[1] / levels[0])
    assert order > p + 1 - 0.35, (errs, order)


@pytest.mark.parametrize("quad", ["LG", "LGL"])
def test_spectral_decay_in_p(quad):
    """At fixed mesh the error falls faster than any fixed power when p grows."""
    sl, st, c = 0.12, 0.03, 1.0

    def exact(x):
        return np.cos(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]) * np.cos(np.pi * x[:, 2])

    errs = []
    s = W.slab(1, 1, 1, (1.0, 1.0, 1.0))
    for p in (2, 4, 6):
        sp_ = Mh.SlabSpace(s.flat_vertices(), 1, 1, 1, p, quad)
        M, K = Mh.assemble_mass_stiffness(sp_, W.constant_tissue(s, sl, st, 0.0))
        f = (np.pi ** 2 * (sl + 2 * st) + c) * exact(sp_.dof_coordinates())
        uh = spla.spsolve((K + c * M).tocsc(), M @ f)
        errs.append(_l2_error(sp_, uh, exact))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs


class _LinearReaction:
    """I_ion = beta u and a frozen gate: isolates the time discretisation."""

    def __init__(self, beta):
        self.beta = beta

    def gate_first(self, h_n, us, dt):
        return h_n

    def gate(self, h_n, h_nm1, us, dt):
        return h_n

    def current(self, us, h):
        return self.beta * us


@pytest.mark.parametrize("quad", ["LG", "LGL"])
def test_bdf2_time_order(quad):
    Lx, sl, beta = 1.0, 0.12, 0.5

    def q(x):
        return x ** 2 * (3 * Lx - 2 * x)

    def d2q(x):
        return 6 * Lx - 12 * x

    def u_exact(t, xyz):
        return (2 + np.sin(np.pi * t)) * q(xyz[:, 0])

    def i_app(t, xyz):
        x = xyz[:, 0]
        return (np.pi * np.cos(np.pi * t) * q(x) + beta * (2 + np.sin(np.pi * t)) * q(x)
                - sl * (2 + np.sin(np.pi * t)) * d2q(x))

    s = W.slab(2, 1, 1, (Lx, 0.5, 0.5))
    sp_ = Mh.SlabSpace(s.flat_vertices(), 2, 1, 1, 3, quad)
    tissue = W.constant_tissue(s, sl, 0.03, 0.0)
    errs = []
    T = 1.0
    for nsteps in (20, 40, 80):
        dt = T / nsteps
        md = MD.Monodomain(sp_, tissue, dt, model=_LinearReaction(beta), i_app_fn=i_app)
        u0 = u_exact(0.0, md.xyz)
        st = dict(u=u0, u_prev=u0.copy(), h=np.zeros_like(u0), h_prev=np.zeros_like(u0), n=0)
        st = md.run(st, nsteps)
        errs.append(np.abs(st["u"] - u_exact(T, md.xyz)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.8 and 3.3 < r2 < 4.8, errs


def test_uniform_state_reduces_to_single_cell():
    """K 1 = 0: a spatially uniform state without stimulus follows the
    single-cell partitioned scheme exactly (same BDF1/BDF2 steps)."""
    from oracle import ionic
    prm = ionic.DEFAULT_PARAMS
    s = W.slab(2, 2, 1, (2.0, 2.0, 1.0), perturb=0.1)
    sp_ = Mh.SlabSpace(s.flat_vertices(), 2, 2, 1, 2, "LG")
    dt = 0.05
    md = MD.Monodomain(sp_, W.constant_tissue(s), dt)
    u0 = np.full(sp_.ndofs, -60.0)
    h0 = np.full(sp_.ndofs, 0.8)
    st = md.run(dict(u=u0, u_prev=u0.copy(), h=h0, h_prev=h0.copy(), n=0), 40)
    ref = ionic.single_cell_semi_implicit(-60.0, 0.8, 40 * dt, dt, prm)
    assert np.abs(st["u"] - ref[0]).max() < 1e-10 * abs(ref[0])
    assert np.abs(st["h"] - ref[1]).max() < 1e-12
