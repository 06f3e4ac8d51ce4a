"""Pins of the oracle's discrete adjoint: central finite differences of the
oracle's own forward loss, and the Taylor remainder of the gradient
(second order in the step)."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD
from oracle import mesh as Mh


def _problem(quad, nsteps=8):
    s = W.slab(3, 2, 1, (3.0, 2.0, 1.0), perturb=0.1, seed=1)
    sp_ = Mh.SlabSpace(s.flat_vertices(), 3, 2, 1, 2, quad)
    ne = s.n_elements
    rng = np.random.default_rng(3)
    tissue = (0.12 * rng.uniform(0.8, 1.2, ne), 0.03 * rng.uniform(0.8, 1.2, ne),
              rng.uniform(-1.0, 1.0, ne))
    sensors = W.seeded_indices(sp_.ndofs, 6, seed=W.SEED_SENSORS)
    model = AD.AdjointModel(sp_, 0.05, nsteps, sensors, region=("box", (0, 0, 0, 1.0, 1.0, 1.0)),
                            amplitude=50.0, t_on=0.0, t_off=0.2)
    u0 = W.uniform_vector(sp_.ndofs, -85.0, -40.0, seed=2)
    h0 = np.full(sp_.ndofs, 0.9)
    tl, tt = W.perturbed_conductivities(tissue[0], tissue[1])
    _, _, target, _ = model.forward((tl, tt, tissue[2]), u0, h0)
    return model, tissue, u0, h0, target


def _loss(model, tissue, u0, h0, target):
    _, _, T, _ = model.forward(tissue, u0, h0)
    return AD.misfit(T, target, model.dt)


@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_adjoint_gradient_matches_central_differences(quad):
    model, tissue, u0, h0, target = _problem(quad)
    L0, Tbar = _loss(model, tissue, u0, h0, target)
    g = model.gradient(tissue, u0, h0, Tbar)
    for k in range(3):
        for e in (0, 2, 5):
            h = 1e-6
            tp = [t.copy() for t in tissue]
            tm = [t.copy() for t in tissue]
            tp[k][e] += h
            tm[k][e] -= h
            fd = (_loss(model, tp, u0, h0, target)[0] - _loss(model, tm, u0, h0, target)[0]) / (2 * h)
            assert abs(g[k][e] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g[k]).max()), (k, e, g[k][e], fd)


def test_adjoint_taylor_remainder_is_second_order():
    model, tissue, u0, h0, target = _problem("LGL", nsteps=6)
    L0, Tbar = _loss(model, tissue, u0, h0, target)
    g = np.concatenate(model.gradient(tissue, u0, h0, Tbar))
    rng = np.random.default_rng(9)
    d = rng.uniform(-1, 1, g.size) * np.concatenate([0.01 * np.ones(6), 0.003 * np.ones(6), 0.1 * np.ones(6)])
    rems = []
    for eps in (1e-2, 5e-3):
        p = np.concatenate(tissue) + eps * d
        tp = (p[:6], p[6:12], p[12:])
        rems.append(abs(_loss(model, tp, u0, h0, target)[0] - L0 - eps * g @ d))
    assert 3.0 < rems[0] / rems[1] < 5.0, rems
