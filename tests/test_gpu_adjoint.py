"""GPU discrete adjoint against the oracle's adjoint gradient and against
central finite differences of the GPU forward model; checkpoint segments of
any length give the same gradient; the torch.autograd.Function returns it."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import adjoint as AD
from oracle import mesh as Mh

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2205_05136_gb300")
capi = gb.capi

BOX = (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)


def _problem(quad, nsteps=8):
    s = W.slab(3, 2, 1, (3.0, 2.0, 1.0), perturb=0.1, seed=1)
    sp_ = Mh.SlabSpace(s.flat_vertices(), 3, 2, 1, 2, quad)
    ne = s.n_elements
    rng = np.random.default_rng(3)
    tissue = (0.12 * rng.uniform(0.8, 1.2, ne), 0.03 * rng.uniform(0.8, 1.2, ne), rng.uniform(-1.0, 1.0, ne))
    sensors = W.seeded_indices(sp_.ndofs, 6, seed=W.SEED_SENSORS)
    model = AD.AdjointModel(sp_, 0.05, nsteps, sensors, region=("box", BOX), amplitude=50.0,
                            t_on=0.0, t_off=0.2)
    u0 = W.uniform_vector(sp_.ndofs, -85.0, -40.0, seed=2)
    h0 = np.full(sp_.ndofs, 0.9)
    tl, tt = W.perturbed_conductivities(tissue[0], tissue[1])
    _, _, target, _ = model.forward((tl, tt, tissue[2]), u0, h0)
    g = gb.Slab(s.flat_vertices(), 3, 2, 1, 2, quad)
    g.set_ionic()
    g.set_stimulus("box", BOX, 50.0, 0.0, 0.2)
    return s, model, tissue, u0, h0, target, sensors, g


def _run(g, tissue, u0, h0, sensors, nsteps, every, target, precond=capi.SEM_PC_JACOBI):
    dev = torch.device("cuda")
    tl = [torch.tensor(t, device=dev, requires_grad=True) for t in tissue]
    T = gb.traces(g, tl[0], tl[1], tl[2], torch.tensor(u0, device=dev), torch.tensor(h0, device=dev),
                  0.05, nsteps, torch.tensor(sensors, dtype=torch.int32), checkpoint_every=every,
                  rtol=1e-13, precond=precond)
    loss = 0.5 * 0.05 * torch.sum((T - torch.tensor(target, device=dev)) ** 2)
    loss.backward()
    return float(loss.detach()), T.detach().cpu().numpy(), [t.grad.cpu().numpy() for t in tl]


@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_adjoint_gradient_matches_oracle(quad):
    s, model, tissue, u0, h0, target, sensors, g = _problem(quad)
    T_ref = model.forward(tissue, u0, h0)[2]
    L_ref, Tbar = AD.misfit(T_ref, target, model.dt)
    ref = np.concatenate(model.gradient(tissue, u0, h0, Tbar))
    for every in (3, 100):
        L, T, grads = _run(g, tissue, u0, h0, sensors, 8, every, target)
        # traces are the forward outputs (1e-10); the misfit loss cancels digits
        assert np.linalg.norm(T - T_ref) < 1e-10 * np.linalg.norm(T_ref)
        assert abs(L - L_ref) < 1e-8 * abs(L_ref)
        got = np.concatenate(grads)
        assert np.linalg.norm(got - ref) < 1e-8 * np.linalg.norm(ref), (every, np.abs(got - ref).max())


def test_adjoint_with_multigrid_solver():
    s, model, tissue, u0, h0, target, sensors, g = _problem("LGL")
    capi.sem_set_gmg(g.ctx, 3, 10, 10, capi.SEM_PREC_FP32)
    L_ref, Tbar = AD.misfit(model.forward(tissue, u0, h0)[2], target, model.dt)
    ref = np.concatenate(model.gradient(tissue, u0, h0, Tbar))
    _, _, grads = _run(g, tissue, u0, h0, sensors, 8, 4, target, precond=capi.SEM_PC_GMG)
    got = np.concatenate(grads)
    assert np.linalg.norm(got - ref) < 1e-8 * np.linalg.norm(ref)


def test_adjoint_matches_gpu_central_differences():
    s, model, tissue, u0, h0, target, sensors, g = _problem("LGL", nsteps=6)
    _, _, grads = _run(g, tissue, u0, h0, sensors, 6, 2, target)
    h = 1e-6
    for k, e in ((0, 1), (1, 4), (2, 0), (2, 3)):
        vals = []
        for sgn in (1, -1):
            tp = [t.copy() for t in tissue]
            tp[k][e] += sgn * h
            L, _, _ = _run(g, tp, u0, h0, sensors, 6, 100, target)
            vals.append(L)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(grads[k][e] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(grads[k]).max()), (k, e, grads[k][e], fd)
