"""GPU parity of the matrix-free operator apply against the CPU oracle.

The CUDA path (through the C ABI) and the oracle (assembled dense element
matrices, Algorithm 2) run on the same seeded inputs.  Tolerance: 1e-12
relative in the 2-norm for FP64 (the operator-apply bound the method's GPU
path is held to); FP32, bf16-metric and tensor-core applies are checked
against error bounds of their precision.
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


# Error bounds of the low-precision applies against the FP64 oracle, each about
# 3x the largest error measured on a GB300 over these cases:
#   FP32 (float u, metric and arithmetic): rounding of u and of the FP32
#     metric, unit roundoff 2^-24 = 6e-8 each; measured <= 1.9e-7 -> 6e-7.
#   bf16 metric: each metric value rounded to bf16, unit roundoff 2^-9 = 2e-3,
#     partly cancelling over a row; measured <= 1.6e-3 -> 5e-3.  The
#     tensor-core kernel (SEM_PREC_BF16_TC) has the same metric and contractions
#     as accurate as FP32 (u, D and q as bf16 hi + lo pairs, 2^-16), so it shares
#     that bound, and it stays within 2e-5 (the pairs' 2^-16 = 1.5e-5; measured
#     <= 5.2e-6) of the scalar bf16-metric kernel.
TOL_FP32, TOL_BF16, TOL_TC_VS_BF16 = 6e-7, 5e-3, 2e-5
LOWP = [(gb.SEM_PREC_FP32, TOL_FP32), (gb.SEM_PREC_FP32_BF16, TOL_BF16), (gb.SEM_PREC_BF16_TC, TOL_BF16)]


def _lowp_cases(prec, quad, p):
    return prec != gb.SEM_PREC_BF16_TC or (quad == "LGL" and 2 <= p <= 4)


@pytest.mark.parametrize("prec,tol", LOWP)
@pytest.mark.parametrize("quad", QUADS)
def test_low_precision_apply_error_bound(prec, tol, quad):
    if not _lowp_cases(prec, quad, 4):
        pytest.skip("the tensor-core apply covers SEM-NI at p = 2..4")
    s = W.slab(4, 3, 2, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
    tissue = _tissue(s)
    g, o = _pair(s, 4, quad, tissue)
    u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=2)
    A = Mh.assemble(o, tissue, 30.0, 1.0)
    y = g.apply(torch.tensor(u, device="cuda", dtype=torch.float32), 30.0, 1.0, precision=prec)
    e = rel(y.double().cpu().numpy(), A @ u)
    assert e < tol, e


@pytest.mark.parametrize("prec,tol", LOWP)
@pytest.mark.parametrize("quad", QUADS)
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_low_precision_apply_ragged_units(p, prec, tol, quad):
    """35 elements: a partial last group of elements in the FP32 kernels at every
    degree (groups of 8, 3, 2, 1 elements per warp at p = 1..4), and units of
    10, 8, 6 elements along x rows of 7 in the tensor-core kernel at p = 2..4."""
    if not _lowp_cases(prec, quad, p):
        pytest.skip("the tensor-core apply covers SEM-NI at p = 2..4")
    s = W.slab(7, 5, 1, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
    tissue = _tissue(s)
    g, o = _pair(s, p, quad, tissue)
    u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=2)
    A = Mh.assemble(o, tissue, 30.0, 1.0)
    y = g.apply(torch.tensor(u, device="cuda", dtype=torch.float32), 30.0, 1.0, precision=prec)
    e = rel(y.double().cpu().numpy(), A @ u)
    assert e < tol, e


@pytest.mark.parametrize("p,dims", [(4, (60, 40, 14)), (3, (80, 40, 16)), (2, (100, 60, 20))])
def test_low_precision_apply_many_units_per_warp(p, dims):
    """Meshes on which every warp of the persistent FP32 kernels runs several
    units, so their cp.async pipelines run many times over (p = 4: 33,600
    elements, about 7 units per warp of the scalar pipelined kernel and 3 per
    warp of the tensor-core kernel): 256 sampled rows against the oracle's
    element rows, and every entry against the FP64 apply."""
    s = W.slab(*dims, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
    tissue = _tissue(s)
    g, o = _pair(s, p, "LGL", tissue)
    u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=2)
    idx = W.seeded_indices(o.ndofs, 256, seed=7)
    ref = Mh.sampled_rows(o, tissue, u, idx, 30.0, 1.0)
    scale = np.abs(ref).max()
    ut = torch.tensor(u, device="cuda")
    y64 = g.apply(ut, 30.0, 1.0)
    assert np.abs(y64.cpu().numpy()[idx] - ref).max() < 1e-12 * scale
    ys = {}
    for prec, tol in LOWP:
        y = g.apply(ut.float(), 30.0, 1.0, precision=prec).double()
        ys[prec] = y
        assert np.abs(y.cpu().numpy()[idx] - ref).max() < tol * scale, prec
        assert rel(y.cpu().numpy(), y64.cpu().numpy()) < tol, prec
    assert rel(ys[gb.SEM_PREC_BF16_TC].cpu().numpy(), ys[gb.SEM_PREC_FP32_BF16].cpu().numpy()) < TOL_TC_VS_BF16
    g.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("p", [2, 3, 4])
def test_tensor_core_apply_matches_scalar_kernel(p):
    """The tensor-core kernel and the scalar FP32 kernel with the same bf16
    metric give the same operator to the accuracy of the bf16 pairs, for
    (alpha, beta) with and without the mass term and with scaling."""
    s = W.slab(13, 4, 3, (20.0, 7.0, 3.0), perturb=0.1, seed=3)
    tissue = _tissue(s)
    g, o = _pair(s, p, "LGL", tissue)
    u = torch.tensor(W.uniform_vector(o.ndofs, -1.0, 1.0, seed=4), device="cuda", dtype=torch.float32)
    for alpha, beta in [(30.0, 1.0), (0.0, 1.0), (2.5, 0.7), (4.0, 0.0)]:
        y = g.apply(u, alpha, beta, precision=gb.SEM_PREC_BF16_TC).double().cpu().numpy()
        yb = g.apply(u, alpha, beta, precision=gb.SEM_PREC_FP32_BF16).double().cpu().numpy()
        assert rel(y, yb) < TOL_TC_VS_BF16, (alpha, beta, rel(y, yb))
    g.close()


def test_tensor_core_apply_reports_unsupported_cases():
    s = W.slab(3, 2, 2, (3.0, 2.0, 1.5), perturb=0.1, seed=21)
    tissue = _tissue(s)
    for p, quad in [(4, "LG"), (1, "LGL"), (5, "LGL")]:
        g, o = _pair(s, p, quad, tissue)
        u = torch.zeros(o.ndofs, dtype=torch.float32, device="cuda")
        y = torch.empty_like(u)
        with pytest.raises(gb.SemError) as ei:
            gb.capi.sem_apply(g.ctx, 30.0, 1.0, u, y, gb.SEM_PREC_BF16_TC)
        assert ei.value.code == gb.capi.SEM_ERR_UNSUPPORTED
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
