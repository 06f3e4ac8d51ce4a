"""GPU parity of the matrix-free operator apply against the CPU oracle.

The CUDA path (through the C ABI) and the oracle (assembled dense element
matrices, Algorithm 2) run on the same seeded inputs.  Tolerance: 1e-12
relative in the 2-norm for FP64 (the operator-apply bound the method's GPU
path is held to); FP32 and bf16-metric applies are checked against error
bounds of their precision.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mesh as Mh

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2205_05136_gb300")

QUADS = ["LG", "LGL"]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _tissue(s, varying=True):
    if not varying:
        return W.constant_tissue(s)
    ne = s.n_elements
    rng = np.random.default_rng(17)
    sl = 0.12 * rng.uniform(0.8, 1.2, ne)
    st = 0.03 * rng.uniform(0.8, 1.2, ne)
    return sl, st, W.transmural_fiber_angles(s)


def _pair(s, p, quad, tissue):
    g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    g.set_tissue(*tissue)
    o = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    return g, o


@pytest.mark.parametrize("quad", QUADS)
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_apply_matches_assembled_operator(p, quad):
    # 3 x 2 x 2 = 12 elements: more than one CTA for p <= 4 and a ragged last CTA
    s = W.slab(3, 2, 2, (3.0, 2.0, 1.5), perturb=0.15, seed=21)
    tissue = _tissue(s)
    g, o = _pair(s, p, quad, tissue)
    assert g.ndofs == o.ndofs
    u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=2)
    M, K = Mh.assemble_mass_stiffness(o, tissue)
    ut = torch.tensor(u, device="cuda")
    for alpha, beta in [(30.0, 1.0), (0.0, 1.0), (1.0, 0.0), (2.5, 0.7)]:
        y = g.apply(ut, alpha, beta).cpu().numpy()
        ref = alpha * (M @ u) + beta * (K @ u)
        assert rel(y, ref) < 1e-12, (alpha, beta, rel(y, ref))


@pytest.mark.parametrize("quad", QUADS)
@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_apply_more_ctas_than_sms(p, quad):
    """A mesh large enough for several waves of CTAs, checked entry by entry."""
    n = {1: (24, 20, 10), 2: (16, 12, 6), 4: (10, 8, 5), 6: (8, 6, 3)}[p]
    s = W.slab(*n, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
    tissue = _tissue(s)
    g, o = _pair(s, p, quad, tissue)
    u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=2)
    A = Mh.assemble(o, tissue, 30.0, 1.0)
    y = g.apply(torch.tensor(u, device="cuda"), 30.0, 1.0).cpu().numpy()
    ref = A @ u
    assert rel(y, ref) < 1e-12
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("quad", QUADS)
@pytest.mark.parametrize("p", [2, 4])
def test_diagonal_and_coords(p, quad):
    s = W.slab(3, 2, 2, (3.0, 2.0, 1.5), perturb=0.15, seed=21)
    tissue = _tissue(s)
    g, o = _pair(s, p, quad, tissue)
    d = g.diagonal(30.0, 1.0).cpu().numpy()
    ref = Mh.diagonal(o, tissue, 30.0, 1.0)
    assert rel(d, ref) < 1e-13
    xyz = g.dof_coords().cpu().numpy().T
    assert np.abs(xyz - o.dof_coordinates()).max() < 1e-13


@pytest.mark.parametrize("quad", QUADS)
def test_single_element_and_thin_slabs(quad):
    for (nx, ny, nz) in [(1, 1, 1), (1, 3, 1), (5, 1, 1)]:
        for p in (1, 3, 6):
            s = W.slab(nx, ny, nz, (1.0, 1.2, 0.8), perturb=0.1 if nx * ny * nz > 1 else 0.0, seed=4)
            tissue = _tissue(s)
            g, o = _pair(s, p, quad, tissue)
            u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=5)
            A = Mh.assemble(o, tissue, 4.0, 1.0)
            y = g.apply(torch.tensor(u, device="cuda"), 4.0, 1.0).cpu().numpy()
            assert rel(y, A @ u) < 1e-12


@pytest.mark.parametrize("prec,tol", [(gb.SEM_PREC_FP32, 2e-6), (gb.SEM_PREC_FP32_BF16, 2e-2)])
@pytest.mark.parametrize("quad", QUADS)
def test_low_precision_apply_error_bound(prec, tol, quad):
    s = W.slab(4, 3, 2, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
    tissue = _tissue(s)
    g, o = _pair(s, 4, quad, tissue)
    u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=2)
    A = Mh.assemble(o, tissue, 30.0, 1.0)
    y = g.apply(torch.tensor(u, device="cuda", dtype=torch.float32), 30.0, 1.0, precision=prec)
    e = rel(y.double().cpu().numpy(), A @ u)
    assert e < tol, e


@pytest.mark.parametrize("prec,tol", [(gb.SEM_PREC_FP32, 2e-6), (gb.SEM_PREC_FP32_BF16, 2e-2)])
@pytest.mark.parametrize("quad", QUADS)
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_low_precision_apply_ragged_units(p, prec, tol, quad):
    """35 elements: a partial last group of elements in the FP32 kernels at every
    degree (groups of 8, 3, 2, 1 elements per warp at p = 1..4)."""
    s = W.slab(7, 5, 1, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
    tissue = _tissue(s)
    g, o = _pair(s, p, quad, tissue)
    u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=2)
    A = Mh.assemble(o, tissue, 30.0, 1.0)
    y = g.apply(torch.tensor(u, device="cuda", dtype=torch.float32), 30.0, 1.0, precision=prec)
    e = rel(y.double().cpu().numpy(), A @ u)
    assert e < tol, e


@pytest.mark.parametrize("prec,tol", [(gb.SEM_PREC_FP32, 2e-6), (gb.SEM_PREC_FP32_BF16, 2e-2)])
@pytest.mark.parametrize("p,dims", [(1, (40, 30, 41)), (2, (37, 30, 25)), (4, (40, 30, 31))])
def test_low_precision_apply_many_groups_per_warp(p, dims, prec, tol):
    """Meshes with several element groups per warp of the persistent FP32 kernel
    (its cp.async pipeline runs over many groups), against the FP64 apply, which
    the oracle checks at every degree."""
    s = W.slab(*dims, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
    g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, "LGL")
    g.set_tissue(*_tissue(s))
    u = torch.tensor(W.uniform_vector(g.ndofs, -1.0, 1.0, seed=2), device="cuda")
    y64 = g.apply(u, 30.0, 1.0)
    y = g.apply(u.float(), 30.0, 1.0, precision=prec).double()
    assert rel(y.cpu().numpy(), y64.cpu().numpy()) < tol
    g.close()


def test_sweep_workload_sampled_rows():
    """Full-size perturbed ~2 M DOF slabs with rotating fibres (the operator
    sweep), in the launch configuration the benchmark times: sampled outputs
    against the oracle's element rows."""
    for p, quad, count in [(4, "LGL", 96), (4, "LG", 96), (1, "LGL", 48), (6, "LG", 24)]:
        s = W.sweep_slab(p)
        tissue = (np.full(s.n_elements, 0.12), np.full(s.n_elements, 0.03), W.transmural_fiber_angles(s))
        g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
        g.set_tissue(*tissue)
        o = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
        u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=W.SEED_U)
        alpha = 1.5 / 0.05
        y = g.apply(torch.tensor(u, device="cuda"), alpha, 1.0).cpu().numpy()
        idx = W.seeded_indices(o.ndofs, count, seed=7)
        ref = Mh.sampled_rows(o, tissue, u, idx, alpha, 1.0)
        scale = np.abs(ref).max()
        assert np.abs(y[idx] - ref).max() < 1e-12 * scale, (p, quad)
        g.close()
        torch.cuda.empty_cache()


@pytest.mark.parametrize("quad", QUADS)
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_df64_apply_matches_assembled_operator(p, quad):
    """Double-float arithmetic on the FP32 pipe meets the FP64 tolerance."""
    s = W.slab(3, 2, 2, (3.0, 2.0, 1.5), perturb=0.15, seed=21)
    tissue = _tissue(s)
    g, o = _pair(s, p, quad, tissue)
    u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=2)
    M, K = Mh.assemble_mass_stiffness(o, tissue)
    ut = torch.tensor(u, device="cuda")
    for alpha, beta in [(30.0, 1.0), (0.0, 1.0), (2.5, 0.7)]:
        y = g.apply(ut, alpha, beta, precision=gb.SEM_PREC_DF64).cpu().numpy()
        ref = alpha * (M @ u) + beta * (K @ u)
        assert rel(y, ref) < 1e-12, (alpha, beta, rel(y, ref))


def test_df64_sweep_workload_sampled_rows():
    for p, quad, count in [(4, "LGL", 64), (4, "LG", 64)]:
        s = W.sweep_slab(p)
        tissue = (np.full(s.n_elements, 0.12), np.full(s.n_elements, 0.03), W.transmural_fiber_angles(s))
        g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
        g.set_tissue(*tissue)
        o = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
        u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=W.SEED_U)
        ut = torch.tensor(u, device="cuda")
        y = g.apply(ut, 30.0, 1.0, precision=gb.SEM_PREC_DF64).cpu().numpy()
        y64 = g.apply(ut, 30.0, 1.0).cpu().numpy()
        idx = W.seeded_indices(o.ndofs, count, seed=7)
        ref = Mh.sampled_rows(o, tissue, u, idx, 30.0, 1.0)
        assert np.abs(y[idx] - ref).max() < 1e-12 * np.abs(ref).max()
        assert rel(y, y64) < 1e-12
        g.close()
        torch.cuda.empty_cache()
