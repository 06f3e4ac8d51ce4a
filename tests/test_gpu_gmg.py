"""GPU parity of the geometric multigrid preconditioner against the oracle's
(Section 4.3): the level hierarchy and its Lanczos eigenvalue estimates, one
V-cycle (FP64: 1e-10; FP32 and bf16-metric: error bounds of their precision),
and the flexible PCG it drives, including time steps against the oracle."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import workloads as W
from oracle import mesh as Mh
from oracle import monodomain as MD
from oracle import multigrid as MG

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2205_05136_gb300")
capi = gb.capi

ALPHA = 1.5 / 0.05


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _setup(dims, p, quad, min_coarse, precision, perturb=0.1):
    s = W.slab(*dims, (20.0, 7.0, 3.0), perturb=perturb, seed=1)
    ne = s.n_elements
    rng = np.random.default_rng(11)
    tissue = (0.12 * rng.uniform(0.8, 1.2, ne), 0.03 * rng.uniform(0.8, 1.2, ne),
              W.transmural_fiber_angles(s))
    g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    g.set_tissue(*tissue)
    capi.sem_set_gmg(g.ctx, 3, 10, min_coarse, precision)
    o = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    H = MG.Hierarchy(o, tissue, ALPHA, degree=3, coarse_degree=10, min_coarse_dofs=min_coarse)
    return s, tissue, g, o, H


@pytest.mark.parametrize("quad", ["LGL", "LG"])
@pytest.mark.parametrize("dims,p,min_coarse", [((6, 4, 3), 4, 30), ((5, 3, 3), 3, 30), ((4, 4, 2), 6, 30),
                                               ((3, 3, 2), 5, 30), ((6, 3, 2), 2, 30),
                                               ((6, 4, 3), 4, 1000)])
def test_hierarchy_and_vcycle_fp64(dims, p, min_coarse, quad):
    s, tissue, g, o, H = _setup(dims, p, quad, min_coarse, capi.SEM_PREC_FP64)
    info = capi.sem_gmg_info(g.ctx, ALPHA)
    assert info["nlevels"] == H.nlevels
    assert info["p"] == [sp_.p for sp_ in H.spaces]
    assert info["dims"] == [(sp_.nx, sp_.ny, sp_.nz) for sp_ in H.spaces]
    assert info["ndofs"] == [sp_.ndofs for sp_ in H.spaces]
    assert np.allclose(info["lambda_max"], H.lam, rtol=1e-10, atol=0)
    r = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=3)
    z = torch.empty(o.ndofs, dtype=torch.float64, device="cuda")
    capi.sem_vcycle(g.ctx, ALPHA, torch.tensor(r, device="cuda"), z)
    ref = H.vcycle(r)
    assert rel(z.cpu().numpy(), ref) < 1e-10


# V-cycle error bounds against the oracle's FP64 V-cycle, about 3x the error
# measured on a GB300: FP32 1.4e-7 (unit roundoff 2^-24 through a few
# applies) -> 5e-7; bf16 metric 1.4e-3 (the metric's 2^-9 rounding) -> 5e-3,
# shared by the tensor-core smoother, whose operator is the bf16-metric one.
@pytest.mark.parametrize("precision,tol", [(capi.SEM_PREC_FP32, 5e-7), (capi.SEM_PREC_FP32_BF16, 5e-3),
                                           (capi.SEM_PREC_BF16_TC, 5e-3)])
def test_vcycle_low_precision_error(precision, tol):
    s, tissue, g, o, H = _setup((6, 4, 3), 4, "LGL", 30, precision)
    r = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=3)
    z = torch.empty(o.ndofs, dtype=torch.float64, device="cuda")
    capi.sem_vcycle(g.ctx, ALPHA, torch.tensor(r, device="cuda"), z)
    e = rel(z.cpu().numpy(), H.vcycle(r))
    assert e < tol, e


@pytest.mark.parametrize("precision", [capi.SEM_PREC_FP32, capi.SEM_PREC_FP32_BF16, capi.SEM_PREC_FP64,
                                       capi.SEM_PREC_BF16_TC])
@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_gmg_pcg_reaches_fp64_solution(precision, quad):
    if precision == capi.SEM_PREC_BF16_TC and quad == "LG":
        with pytest.raises(gb.SemError):
            _setup((8, 5, 3), 4, quad, 200, precision)
        return
    s, tissue, g, o, H = _setup((8, 5, 3), 4, quad, 200, precision)
    A = H.A[0]
    b = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=5)
    xref = spla.spsolve(A.tocsc(), b)
    x = torch.zeros(o.ndofs, dtype=torch.float64, device="cuda")
    it, res = g.cg_solve(ALPHA, torch.tensor(b, device="cuda"), x, rtol=1e-13, maxit=200,
                         precond=capi.SEM_PC_GMG)
    assert rel(x.cpu().numpy(), xref) < 1e-10
    assert it <= 20, it
    # the oracle's flexible PCG with the same V-cycle needs a similar count
    _, it_ref = H.pcg(b, rtol=1e-13)
    assert abs(it - it_ref) <= 3, (it, it_ref)


@pytest.mark.parametrize("offset", [0, 1])
def test_gmg_pcg_double_float_operator(offset):
    """The flexible PCG with the double-float operator (its vector kernels move
    two entries at a time with 16-byte accesses): an odd node count (9009) for
    the one-entry tail, and with offset 1 a solution and right-hand side that
    start 8 bytes past a 16-byte boundary, which the kernels take one entry at a
    time.  Both reach the direct solution."""
    s, tissue, g, o, H = _setup((8, 5, 3), 4, "LGL", 200, capi.SEM_PREC_FP32_BF16)
    capi.sem_set_operator_precision(g.ctx, capi.SEM_PREC_DF64)
    assert o.ndofs % 2 == 1
    A = H.A[0]
    b = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=5)
    xref = spla.spsolve(A.tocsc(), b)
    bb = torch.zeros(o.ndofs + offset, dtype=torch.float64, device="cuda")[offset:]
    bb.copy_(torch.tensor(b))
    x = torch.zeros(o.ndofs + offset, dtype=torch.float64, device="cuda")[offset:]
    assert (x.data_ptr() % 16 == 8) == (offset == 1) and (bb.data_ptr() % 16 == 8) == (offset == 1)
    it, res = g.cg_solve(ALPHA, bb, x, rtol=1e-12, maxit=200, precond=capi.SEM_PC_GMG)
    assert rel(x.cpu().numpy(), xref) < 1e-10
    assert it <= 20, it


@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_time_steps_with_fp32_multigrid_match_oracle(quad):
    s = W.slab(8, 4, 2, (20.0, 7.0, 3.0))
    tissue = W.constant_tissue(s, 0.12, 0.03, 0.0)
    g = gb.Slab(s.flat_vertices(), 8, 4, 2, 2, quad)
    g.set_tissue(*tissue)
    capi.sem_set_gmg(g.ctx, 3, 10, 100, capi.SEM_PREC_FP32)
    box = (0.0, 0.0, 0.0, 1.5, 1.5, 1.5)
    g.set_ionic()
    g.set_stimulus("box", box, 50.0, 0.0, 1.0)
    st = g.new_state(-85.0, 1.0)
    stats = st.step(0.05, 40, rtol=1e-13, maxit=500, precond=capi.SEM_PC_GMG)
    u, h, n = st.get()
    o = Mh.SlabSpace(s.flat_vertices(), 8, 4, 2, 2, quad)
    md = MD.Monodomain(o, tissue, 0.05, region=("box", box), amplitude=50.0, t_on=0.0, t_off=1.0)
    ref = md.run(MD.rest_state(o.ndofs), 40)
    assert n == 40
    assert rel(u.cpu().numpy(), ref["u"]) < 1e-10
    assert stats.cg_iters / 40 < 12
