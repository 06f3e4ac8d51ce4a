"""The SEM_DEBUG build: index checks in the apply and transfer kernels.

That build checks every node index the kernels take from the element-to-DOF map
against [0, ndofs), records the first one outside in a device word instead of
using it (node 0 is used), and the host returns SEM_ERR_ARG naming it.  The test
builds the variant (libsem_debug.so), runs it in a child process selected by
SEM_LIBRARY, plants an out-of-range entry in the map through
sem_debug_set_map_entry, and checks that the FP64 apply, the FP32 smoother
apply, a multigrid V-cycle and a CG solve all report it; with the entry
restored the results are again those of the clean run.  The same child also
holds back one metric copy of the pipelined apply (sem_debug_hold_copy): the
bounded wait for it runs out and the multigrid solve returns SEM_ERR_TIMEOUT,
after which the context solves as before.  The normal build answers both
debug entry points with SEM_ERR_UNSUPPORTED.
"""
import os
import subprocess
import sys

import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2205_05136_gb300")
capi = gb.capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import workloads as W
from paper_2205_05136_gb300 import capi
import paper_2205_05136_gb300 as gb
assert "SEM_DEBUG" in capi.sem_version(), capi.sem_version()
s = W.slab(5, 4, 3, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, 4, "LGL")
g.set_tissue(np.full(s.n_elements, 0.12), np.full(s.n_elements, 0.03), W.transmural_fiber_angles(s))
capi.sem_set_gmg(g.ctx, 3, 10, 100, capi.SEM_PREC_FP32_BF16)
u = torch.tensor(W.uniform_vector(g.ndofs, -1.0, 1.0, seed=2), device="cuda")
y0 = g.apply(u, 30.0, 1.0)
y0f = g.apply(u.float(), 30.0, 1.0, precision=capi.SEM_PREC_FP32_BF16)
z0 = torch.empty_like(u)
capi.sem_vcycle(g.ctx, 30.0, u, z0)
bad = g.ndofs + 3
entry = 2 * 125 + 37          # element 2, local node 37
old = capi.sem_debug_set_map_entry(g.ctx, entry, bad)
def expect_error(fn, what):
    try:
        fn()
    except capi.SemError as e:
        assert e.code == capi.SEM_ERR_ARG, (what, e.code)
        assert str(bad) in str(e) and "SEM_DEBUG" in str(e), (what, str(e))
        return
    raise AssertionError(what + ": no SEM_DEBUG error")
expect_error(lambda: g.apply(u, 30.0, 1.0), "fp64 apply")
expect_error(lambda: g.apply(u.float(), 30.0, 1.0, precision=capi.SEM_PREC_FP32_BF16), "bf16 apply")
expect_error(lambda: capi.sem_vcycle(g.ctx, 30.0, u, torch.empty_like(u)), "v-cycle")
x = torch.zeros_like(u)
expect_error(lambda: capi.sem_cg_solve(g.ctx, 30.0, u, x, 1e-10, 0.0, 50, capi.SEM_PC_JACOBI), "cg")
assert capi.sem_debug_set_map_entry(g.ctx, entry, old) == bad
y1 = g.apply(u, 30.0, 1.0)
assert float(torch.linalg.norm(y1 - y0) / torch.linalg.norm(y0)) < 1e-14
y1f = g.apply(u.float(), 30.0, 1.0, precision=capi.SEM_PREC_FP32_BF16)
assert float(torch.linalg.norm(y1f - y0f) / torch.linalg.norm(y0f)) < 1e-6
z1 = torch.empty_like(u)
capi.sem_vcycle(g.ctx, 30.0, u, z1)
assert float(torch.linalg.norm(z1 - z0) / torch.linalg.norm(z0)) < 1e-6
# the timeout path: the fine level's pipelined apply leaves out the metric copy of
# element group 3, the wait for it runs out, the multigrid solve reports it, and
# the context then solves as before
xr = torch.zeros_like(u)
capi.sem_cg_solve(g.ctx, 30.0, u, xr, 1e-10, 0.0, 100, capi.SEM_PC_GMG)
capi.sem_debug_hold_copy(g.ctx, 3)
try:
    capi.sem_cg_solve(g.ctx, 30.0, u, torch.zeros_like(u), 1e-10, 0.0, 100, capi.SEM_PC_GMG)
    raise AssertionError("no timeout reported")
except capi.SemError as e:
    assert e.code == capi.SEM_ERR_TIMEOUT, (e.code, str(e))
capi.sem_debug_hold_copy(g.ctx, -1)
x2 = torch.zeros_like(u)
capi.sem_cg_solve(g.ctx, 30.0, u, x2, 1e-10, 0.0, 100, capi.SEM_PC_GMG)
assert float(torch.linalg.norm(x2 - xr) / torch.linalg.norm(xr)) < 1e-12
g.close()
print("debug build ok")
"""


def test_debug_build_reports_planted_map_index():
    from paper_2205_05136_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ)
    env["SEM_LIBRARY"] = lib
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug build ok" in r.stdout


def test_normal_build_has_no_map_fault_injection():
    s = W.slab(2, 2, 1, (2.0, 2.0, 1.0))
    g = gb.Slab(s.flat_vertices(), 2, 2, 1, 2, "LGL")
    assert "SEM_DEBUG" not in capi.sem_version()
    with pytest.raises(capi.SemError) as ei:
        capi.sem_debug_set_map_entry(g.ctx, 0, 5)
    assert ei.value.code == capi.SEM_ERR_UNSUPPORTED
    with pytest.raises(capi.SemError) as ei:
        capi.sem_debug_hold_copy(g.ctx, 0)
    assert ei.value.code == capi.SEM_ERR_UNSUPPORTED
    u = torch.zeros(g.ndofs, dtype=torch.float64, device="cuda")
    g.apply(u, 1.0, 1.0)  # the context is unaffected
    g.close()
