"""Differentiable sensor traces of the monodomain time stepping.

``traces(slab, sigma_l, sigma_t, theta, u0, h0, dt, nsteps, sensors, ...)``
runs the forward time steps in libsem (sem_forward_record) and returns the
potential at the sensor nodes after every step, T[k, s].  Its backward pass
calls libsem's discrete adjoint (sem_adjoint_grad), which recomputes each
checkpoint segment and returns dL/dsigma_l, dL/dsigma_t, dL/dtheta per
element for any loss L(T).  Both directions run entirely in the CUDA library.
"""
from __future__ import annotations

import torch

from . import capi


class _Traces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_l, sigma_t, theta, slab, u0, h0, dt, nsteps, sensors, every, solver):
        rtol, atol, maxit, precond = solver
        slab.set_tissue(sigma_l.detach(), sigma_t.detach(), theta.detach())
        st = slab.new_state(u0, h0)
        sens = sensors.to(device=slab.device, dtype=torch.int32).contiguous()
        T = torch.empty(nsteps, sens.numel(), dtype=torch.float64, device=slab.device)
        capi.sem_forward_record(slab.ctx, st._st, dt, nsteps, every, sens, T, rtol, atol, maxit, precond)
        st.close()
        slab._recording = getattr(slab, "_recording", 0) + 1
        ctx.slab = slab
        ctx.recording = slab._recording
        ctx.solver = solver
        ctx.save_for_backward(sigma_l.detach(), sigma_t.detach(), theta.detach())
        return T

    @staticmethod
    def backward(ctx, grad_T):
        slab = ctx.slab
        if slab._recording != ctx.recording:
            raise RuntimeError("a later forward run replaced the recording this backward needs")
        rtol, atol, maxit, precond = ctx.solver
        sl, st_, th = ctx.saved_tensors
        slab.set_tissue(sl, st_, th)  # the adjoint needs the recording's tissue
        g = [torch.empty(slab.nelem, dtype=torch.float64, device=slab.device) for _ in range(3)]
        capi.sem_adjoint_grad(slab.ctx, grad_T.to(torch.float64).contiguous(), g[0], g[1], g[2], rtol,
                              atol, maxit, precond)
        return g[0], g[1], g[2], None, None, None, None, None, None, None, None


def traces(slab, sigma_l, sigma_t, theta, u0, h0, dt, nsteps, sensors, checkpoint_every=20,
           rtol=1e-10, atol=0.0, maxit=2000, precond=capi.SEM_PC_JACOBI):
    """Sensor traces T[k, s] = u^{k+1}[sensors[s]], differentiable in the tissue."""
    return _Traces.apply(sigma_l, sigma_t, theta, slab, u0, h0, float(dt), int(nsteps), sensors,
                         int(checkpoint_every), (float(rtol), float(atol), int(maxit), int(precond)))
