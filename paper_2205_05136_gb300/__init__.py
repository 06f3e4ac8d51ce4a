"""GB300-native matrix-free SEM / SEM-NI monodomain solver (arXiv 2205.05136).

The compute lives in ``libsem.so`` (CUDA C++ for sm_103a behind the C ABI of
``include/sem.h``); this package is its Python binding:

* ``capi``  -- one ctypes wrapper per C entry point, same names;
* ``Slab``  -- a context (mesh, metric terms, solver) on one device;
* ``build`` -- compiles the library in-tree.

PyTorch supplies device memory and streams.  There is no CPU fallback: if
libsem.so is missing, using the package raises.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi
from .autograd import traces  # noqa: F401
from .capi import (SEM_PC_GMG, SEM_PC_JACOBI, SEM_PC_NONE, SEM_PREC_BF16_TC, SEM_PREC_DF64, SEM_PREC_FP32,  # noqa: F401
                   SEM_PREC_FP32_BF16,
                   SEM_PREC_FP64, SEM_QUAD_LG, SEM_QUAD_LGL, SEM_REGION_BOX, SEM_REGION_SPHERE,
                   SemError)

QUAD = {"LG": SEM_QUAD_LG, "SEM": SEM_QUAD_LG, "LGL": SEM_QUAD_LGL, "SEM-NI": SEM_QUAD_LGL}

DEFAULT_IONIC = dict(u_rest=-85.0, u_amp=100.0, tau_in=0.3, tau_out=6.0, tau_open=120.0,
                     tau_close=150.0, v_gate=0.13, kappa=0.01)


class Slab:
    """A libsem context for a structured slab of nx x ny x nz Q_p hexahedra.

    vertices: float64 array of (nx+1)(ny+1)(nz+1) points (x fastest).
    quad: "LG" (SEM) or "LGL" (SEM-NI).
    """

    def __init__(self, vertices, nx: int, ny: int, nz: int, p: int, quad="LGL", device: int = 0):
        self.device = torch.device("cuda", device)
        self.nx, self.ny, self.nz, self.p = nx, ny, nz, p
        self.quad = QUAD[quad] if isinstance(quad, str) else int(quad)
        self._ctx = capi.sem_create(nx, ny, nz, np.asarray(vertices, dtype=np.float64), p,
                                    self.quad, device)
        self.ndofs = capi.sem_num_dofs(self._ctx)
        self.nelem = capi.sem_num_elements(self._ctx)

    @property
    def ctx(self):
        return self._ctx

    def close(self):
        if getattr(self, "_ctx", None) is not None:
            capi.sem_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, dtype=torch.float64):
        return torch.empty(self.ndofs, dtype=dtype, device=self.device)

    def dof_coords(self) -> torch.Tensor:
        xyz = torch.empty(3, self.ndofs, dtype=torch.float64, device=self.device)
        capi.sem_dof_coords(self._ctx, xyz)
        return xyz

    def set_tissue(self, sigma_l, sigma_t, theta):
        f = lambda a: torch.as_tensor(a, dtype=torch.float64).to(self.device).contiguous()  # noqa: E731
        capi.sem_set_tissue(self._ctx, f(sigma_l), f(sigma_t), f(theta))

    def apply(self, u: torch.Tensor, alpha=1.0, beta=1.0, precision=SEM_PREC_FP64, out=None):
        dt = torch.float64 if precision in (SEM_PREC_FP64, SEM_PREC_DF64) else torch.float32
        y = out if out is not None else self._vec(dt)
        capi.sem_apply(self._ctx, alpha, beta, u, y, precision)
        return y

    def diagonal(self, alpha=1.0, beta=1.0):
        d = self._vec()
        capi.sem_diagonal(self._ctx, alpha, beta, d)
        return d

    def cg_solve(self, alpha, b, x, rtol=1e-10, atol=0.0, maxit=1000, precond=SEM_PC_JACOBI):
        _, it, res = capi.sem_cg_solve(self._ctx, alpha, b, x, rtol, atol, maxit, precond)
        return it, res

    def set_ionic(self, **params):
        prm = dict(DEFAULT_IONIC)
        prm.update(params)
        capi.sem_set_ionic(self._ctx, prm)

    def set_stimulus(self, region, params, amplitude, t_on, t_off):
        r = {"box": SEM_REGION_BOX, "sphere": SEM_REGION_SPHERE}.get(region, region)
        capi.sem_set_stimulus(self._ctx, r, params, amplitude, t_on, t_off)

    def new_state(self, u0, h0):
        return State(self, u0, h0)

    def set_timing(self, enable=True):
        capi.sem_set_timing(self._ctx, enable)


class State:
    """BDF2 time-stepping state (u^n, u^{n-1}, h^n, h^{n-1}, n) on the device."""

    def __init__(self, slab: Slab, u0, h0):
        self.slab = slab
        self._st = capi.sem_state_create(slab.ctx)
        self.set(u0, h0)

    def set(self, u0, h0):
        s = self.slab
        u0 = torch.as_tensor(u0, dtype=torch.float64).to(s.device).contiguous()
        h0 = torch.as_tensor(h0, dtype=torch.float64).to(s.device).contiguous()
        if u0.numel() == 1:
            u0 = u0.expand(s.ndofs).contiguous()
        if h0.numel() == 1:
            h0 = h0.expand(s.ndofs).contiguous()
        capi.sem_state_set(s.ctx, self._st, u0, h0)

    def get(self):
        """(u^n, h^n, n)."""
        s = self.slab
        u = s._vec()
        h = s._vec()
        n = capi.sem_state_get(s.ctx, self._st, u=u, h=h)
        return u, h, n

    def checkpoint(self):
        """Full BDF2 state: dict(u, u_prev, h, h_prev, n) as device tensors."""
        s = self.slab
        out = {k: s._vec() for k in ("u", "u_prev", "h", "h_prev")}
        out["n"] = capi.sem_state_get(s.ctx, self._st, **out)
        return out

    def restore(self, ck):
        capi.sem_state_restore(self.slab.ctx, self._st, ck["u"], ck["u_prev"], ck["h"],
                               ck["h_prev"], ck["n"])

    def step(self, dt, nsteps=1, rtol=1e-10, atol=0.0, maxit=1000, precond=SEM_PC_JACOBI):
        return capi.sem_step(self.slab.ctx, self._st, dt, nsteps, rtol, atol, maxit, precond)

    def track_activation(self, enable=True):
        """Record activation times (Eq. tau) from the next step on (enabling resets them)."""
        capi.sem_state_track_activation(self.slab.ctx, self._st, enable)

    def activation(self):
        """(tau, max |du/dt|) per node as device tensors: the time of the step with the
        largest |du/dt| so far and that value."""
        s = self.slab
        tau, dmax = s._vec(), s._vec()
        capi.sem_state_get_activation(s.ctx, self._st, tau, dmax)
        return tau, dmax

    def close(self):
        if getattr(self, "_st", None) is not None:
            capi.sem_state_destroy(self._st)
            self._st = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Slab", "State", "capi", "SemError", "QUAD", "DEFAULT_IONIC", "traces"]
