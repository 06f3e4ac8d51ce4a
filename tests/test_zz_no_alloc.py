"""The allocation-free apply (sem_apply_dot_static) against the regular apply.

sem_apply_dot_static serves callers that cannot let a library allocate device
memory (hosts that own every device allocation through their own arena or
budget, loops that must not enter the allocator): its reduction scratch is a
static device array inside libsem.  This test calls it through the C ABI twice
in a row, with different inputs, and checks y against sem_apply's output and
against the oracle's assembled operator, and the returned u . y against the
inner product of u with those outputs.  It lives in its own file, collected
last, and passes alone in a fresh process or after the other tests.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mesh as Mh

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2205_05136_gb300")
capi = gb.capi

DIMS = (12, 9, 5)


def _slab(p, dims, quad="LGL", fibres=True):
    s = W.slab(*dims, (20.0, 7.0, 3.0), perturb=0.1 if fibres else 0.0, seed=1)
    g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    tissue = None
    if fibres:
        ne = s.n_elements
        tissue = (np.full(ne, 0.12), np.full(ne, 0.03), W.transmural_fiber_angles(s))
        g.set_tissue(*tissue)
    return s, g, tissue


@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_static_scratch_apply_matches_sem_apply_twice(quad):
    from paper_2205_05136_gb300 import build
    build.build()
    s, g, tissue = _slab(3, DIMS, quad)
    o = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, 3, quad)
    M, K = Mh.assemble_mass_stiffness(o, tissue)
    for seed, (a, b) in ((2, (30.0, 1.0)), (3, (2.5, 0.7))):
        un = W.uniform_vector(g.ndofs, -1.0, 1.0, seed=seed)
        u = torch.tensor(un, device="cuda")
        y_ref = torch.empty_like(u)
        capi.sem_apply(g.ctx, a, b, u, y_ref)
        y = torch.full_like(u, float("nan"))
        dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        capi.sem_apply_dot_static(g.ctx, a, b, u, y, dot)
        torch.cuda.synchronize()
        # the existing entry point
        err = float(torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref))
        assert err < 1e-12, err
        ref_dot = float(torch.dot(u, y_ref))
        assert abs(float(dot[0]) - ref_dot) < 1e-12 * abs(ref_dot)
        # the oracle's assembled operator
        yo = a * (M @ un) + b * (K @ un)
        yn = y.cpu().numpy()
        assert np.linalg.norm(yn - yo) < 1e-12 * np.linalg.norm(yo)
        assert abs(float(dot[0]) - float(un @ yo)) < 1e-12 * abs(float(un @ yo))
    g.close()


def test_static_scratch_rejects_overlapping_outputs():
    _, g, _ = _slab(2, (3, 2, 2))
    u = torch.zeros(g.ndofs + 1, dtype=torch.float64, device="cuda")
    y = torch.empty(g.ndofs, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.SemError) as ei:   # dot inside y
        capi.sem_apply_dot_static(g.ctx, 1.0, 1.0, u[: g.ndofs], y, y[3:4])
    assert ei.value.code == capi.SEM_ERR_ARG
    with pytest.raises(capi.SemError) as ei:   # y shifted by one entry over u
        capi.sem_apply_dot_static(g.ctx, 1.0, 1.0, u[: g.ndofs], u[1:], y[:1])
    assert ei.value.code == capi.SEM_ERR_ARG
    g.close()


def test_static_scratch_rejects_meshes_beyond_its_size():
    # p = 1: 64 elements per CTA, so 65,536 CTAs cover 4,194,304 elements
    _, g, _ = _slab(1, (160, 160, 165), fibres=False)
    assert g.nelem > 65536 * 64
    u = torch.zeros(g.ndofs, dtype=torch.float64, device="cuda")
    y = torch.empty_like(u)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.SemError) as ei:
        capi.sem_apply_dot_static(g.ctx, 1.0, 1.0, u, y, dot)
    assert ei.value.code == capi.SEM_ERR_ARG
    assert "static scratch" in str(ei.value)
    g.close()
