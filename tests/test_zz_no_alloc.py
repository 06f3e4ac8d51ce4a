"""The allocation-free apply (sem_apply_dot_static) against the regular apply.

sem_apply_dot_static serves callers that cannot allocate device memory (for
example code running under CUDA stream capture, or hosts that own every
device allocation): its reduction scratch is a static device array inside
libsem.  This test calls it through the C ABI twice in a row, with different
inputs, and checks y against sem_apply's output and the returned u . y
against the inner product of u with that output.  It lives in its own file,
collected last, and passes alone in a fresh process or after the other tests.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2205_05136_gb300")
capi = gb.capi


def _slab(p, dims, quad="LGL", fibres=True):
    s = W.slab(*dims, (20.0, 7.0, 3.0), perturb=0.1 if fibres else 0.0, seed=1)
    g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    if fibres:
        ne = s.n_elements
        g.set_tissue(np.full(ne, 0.12), np.full(ne, 0.03), W.transmural_fiber_angles(s))
    return g


@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_static_scratch_apply_matches_sem_apply_twice(quad):
    from paper_2205_05136_gb300 import build
    build.build()
    g = _slab(3, (12, 9, 5), quad)
    alpha, beta = 30.0, 1.0
    for seed, (a, b) in ((2, (alpha, beta)), (3, (2.5, 0.7))):
        u = torch.tensor(W.uniform_vector(g.ndofs, -1.0, 1.0, seed=seed), device="cuda")
        y_ref = torch.empty_like(u)
        capi.sem_apply(g.ctx, a, b, u, y_ref)
        y = torch.full_like(u, float("nan"))
        dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        capi.sem_apply_dot_static(g.ctx, a, b, u, y, dot)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref))
        assert err < 1e-12, err
        ref_dot = float(torch.dot(u, y_ref))
        assert abs(float(dot[0]) - ref_dot) < 1e-12 * abs(ref_dot)
    g.close()


def test_static_scratch_rejects_meshes_beyond_its_size():
    # p = 1: 64 elements per CTA, so 65,536 CTAs cover 4,194,304 elements
    g = _slab(1, (160, 160, 165), fibres=False)
    assert g.nelem > 65536 * 64
    u = torch.zeros(g.ndofs, dtype=torch.float64, device="cuda")
    y = torch.empty_like(u)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.SemError) as ei:
        capi.sem_apply_dot_static(g.ctx, 1.0, 1.0, u, y, dot)
    assert ei.value.code == capi.SEM_ERR_ARG
    assert "static scratch" in str(ei.value)
    g.close()
