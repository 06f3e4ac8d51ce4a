"""Deterministic mode (sem_set_deterministic): bitwise reproducible results.

The element results of an apply are normally scatter-added with atomics, whose
order varies between runs.  In deterministic mode they go to element-local
storage and a node kernel adds each node's contributions in a fixed order
(Algorithm 1's "compress" step done as a gather).  These tests run the apply,
the multigrid V-cycle (p- and h-restrictions included), a multigrid PCG solve
and time steps twice on the same inputs and compare bitwise, and check the
results against the oracle with the tolerances of the other parity tests.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mesh as Mh
from oracle import multigrid as MG

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2205_05136_gb300")
capi = gb.capi

ALPHA = 1.5 / 0.05


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _slab(dims, p, quad, seed=11):
    s = W.slab(*dims, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
    ne = s.n_elements
    rng = np.random.default_rng(seed)
    tissue = (0.12 * rng.uniform(0.8, 1.2, ne), 0.03 * rng.uniform(0.8, 1.2, ne),
              W.transmural_fiber_angles(s))
    g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    g.set_tissue(*tissue)
    return s, tissue, g


@pytest.mark.parametrize("quad", ["LGL", "LG"])
@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_apply_bitwise_reproducible(p, quad):
    dims = {1: (20, 12, 9), 2: (12, 8, 5), 4: (9, 7, 4), 6: (6, 4, 3)}[p]
    s, tissue, g = _slab(dims, p, quad)
    capi.sem_set_deterministic(g.ctx, True)
    o = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    u = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=2)
    ut = torch.tensor(u, device="cuda")
    precs = [(gb.SEM_PREC_FP64, torch.float64), (gb.SEM_PREC_DF64, torch.float64),
             (gb.SEM_PREC_FP32, torch.float32), (gb.SEM_PREC_FP32_BF16, torch.float32)]
    for prec, dt in precs:
        for alpha, beta in [(ALPHA, 1.0), (2.5, 0.7), (1.0, 0.0)]:
            y1 = g.apply(ut.to(dt), alpha, beta, precision=prec)
            y2 = g.apply(ut.to(dt), alpha, beta, precision=prec)
            assert torch.equal(y1, y2), (prec, alpha, beta)
    # the deterministic FP64 apply is the same operator: the oracle's tolerance
    idx = W.seeded_indices(o.ndofs, 48, seed=7)
    ref = Mh.sampled_rows(o, tissue, u, idx, ALPHA, 1.0)
    y = g.apply(ut, ALPHA, 1.0).cpu().numpy()
    assert np.abs(y[idx] - ref).max() < 1e-12 * np.abs(ref).max()
    g.close()


def test_tensor_core_apply_reports_no_deterministic_mode():
    s, tissue, g = _slab((6, 4, 3), 4, "LGL")
    capi.sem_set_deterministic(g.ctx, True)
    u = torch.zeros(g.ndofs, dtype=torch.float32, device="cuda")
    with pytest.raises(gb.SemError) as ei:
        capi.sem_apply(g.ctx, ALPHA, 1.0, u, torch.empty_like(u), gb.SEM_PREC_BF16_TC)
    assert ei.value.code == capi.SEM_ERR_UNSUPPORTED
    g.close()


@pytest.mark.parametrize("precision", [capi.SEM_PREC_FP64, capi.SEM_PREC_FP32_BF16, capi.SEM_PREC_BF16_TC])
def test_vcycle_with_h_levels_reproducible_and_parity(precision):
    """p 4 -> 2 -> 1, then h-levels (8 x 6 x 4 -> 4 x 3 x 2 -> 2 x 2 x 1): every
    restriction runs in its deterministic form."""
    s, tissue, g = _slab((8, 6, 4), 4, "LGL")
    capi.sem_set_deterministic(g.ctx, True)
    capi.sem_set_gmg(g.ctx, 3, 10, 30, precision)
    info = capi.sem_gmg_info(g.ctx, ALPHA)
    assert info["p"][:3] == [4, 2, 1] and info["nlevels"] >= 4  # h-levels are present
    o = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, 4, "LGL")
    H = MG.Hierarchy(o, tissue, ALPHA, degree=3, coarse_degree=10, min_coarse_dofs=30)
    r = torch.tensor(W.uniform_vector(o.ndofs, -1.0, 1.0, seed=3), device="cuda")
    z1 = torch.empty_like(r)
    z2 = torch.empty_like(r)
    capi.sem_vcycle(g.ctx, ALPHA, r, z1)
    capi.sem_vcycle(g.ctx, ALPHA, r, z2)
    assert torch.equal(z1, z2)
    tol = 1e-10 if precision == capi.SEM_PREC_FP64 else 5e-3
    assert rel(z1.cpu().numpy(), H.vcycle(r.cpu().numpy())) < tol
    g.close()


def test_mixed_gmg_time_steps_bitwise_reproducible():
    """The benchmark's solver (df64 outer operator, bf16-metric V-cycle) on a
    stimulated slab: 8 time steps twice from the same state give bitwise the
    same u and h, and match the atomic-scatter run to the solver tolerance."""
    s, tissue, g = _slab((10, 6, 4), 4, "LGL")
    g.set_ionic()
    g.set_stimulus("box", (0.0, 0.0, 0.0, 4.0, 3.0, 1.5), 50.0, 0.0, 1.0)
    capi.sem_set_operator_precision(g.ctx, gb.SEM_PREC_DF64)
    capi.sem_set_gmg(g.ctx, 6, 5, 2000, gb.SEM_PREC_FP32_BF16)
    out = []
    for det in (True, True, False):
        capi.sem_set_deterministic(g.ctx, det)
        st = g.new_state(-85.0, 1.0)
        st.step(0.05, 8, rtol=1e-12, maxit=200, precond=gb.SEM_PC_GMG)
        u, h, n = st.get()
        out.append((u.clone(), h.clone()))
        st.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert float(out[0][0].max()) > -84.0  # the stimulus acted
    assert rel(out[0][0].cpu().numpy(), out[2][0].cpu().numpy()) < 1e-10
    g.close()
