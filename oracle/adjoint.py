"""Oracle: discrete adjoint of the partitioned time stepping (test infrastructure).

Part of the CPU oracle (plain float64, never called by the product path).

The forward map is the scheme of ``oracle.monodomain`` (Section 3, Eqs.
(ionic_discr)-(matrix_rhs); BDF1 first step, BDF2 afterwards) with the
stand-in ionic model.  Observed quantities are "traces": the potential at a
set of sensor nodes after every step, T[n, s] = u^{n+1}_{sensor_s}
(n = 0 .. N-1).  For a loss L(T) with dL/dT given, this module returns the
gradient of L with respect to the per-element conductivities sigma_l,
sigma_t and fibre angle theta, which enter only through the stiffness
matrix K = sum_e K_e with D_e = sigma_t I + (sigma_l - sigma_t) f f^T,
f = (cos theta, sin theta, 0):

  dD/dsigma_l = f f^T,   dD/dsigma_t = I - f f^T,
  dD/dtheta   = (sigma_l - sigma_t) (f' f^T + f f'^T),  f' = (-sin, cos, 0).

Discrete adjoint, reverse over the steps n = N-1 .. 0 (A_n = alpha_n M + K):
  w        = A_n^{-1} ubar^{n+1}                 (A symmetric)
  grad_e  -= w_e^T K_e[dD] u_e^{n+1}              (each parameter)
  gbar     = M w
  BDF2:  ubar^n += (2/dt) gbar,  ubar^{n-1} -= gbar / (2 dt)
  BDF1:  ubar^0 += gbar / dt
  Ibar     = -gbar
  ustarbar = Ibar dI/du*,   hbar^{n+1} += Ibar dI/dh
  ustarbar += hbar^{n+1} dh^{n+1}/du*
  BDF2:  hbar^n += 4 hbar^{n+1} / D,  hbar^{n-1} -= hbar^{n+1} / D,
         ubar^n += 2 ustarbar,  ubar^{n-1} -= ustarbar
  BDF1:  hbar^0 += hbar^{n+1} / D1,  ubar^0 += ustarbar
with the trace sensitivities added to ubar^{n+1} before step n is reversed.
The loss used by the tests (the workloads' reading) is the sensor misfit
L = dt/2 sum_n sum_s (T[n, s] - target[n, s])^2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import ionic
from .element import diffusion_tensor, element_matrices
from .mesh import SlabSpace
from .monodomain import region_indicator


def _tissue_tensors(sl, st, th):
    f = np.array([np.cos(th), np.sin(th), 0.0])
    fp = np.array([-np.sin(th), np.cos(th), 0.0])
    ff = np.outer(f, f)
    return ff, np.eye(3) - ff, (sl - st) * (np.outer(fp, f) + np.outer(f, fp))


class AdjointModel:
    """Forward traces and their adjoint gradient on a small slab (assembled
    matrices, exact sparse solves)."""

    def __init__(self, space: SlabSpace, dt: float, nsteps: int, sensors, params=None,
                 region=None, amplitude=0.0, t_on=0.0, t_off=0.0):
        self.space, self.dt, self.nsteps = space, float(dt), int(nsteps)
        self.sensors = np.asarray(sensors, dtype=np.int64)
        self.prm = dict(ionic.DEFAULT_PARAMS if params is None else params)
        self.amplitude, self.t_on, self.t_off = amplitude, t_on, t_off
        self.mask = (region_indicator(space.dof_coordinates(), region) if region is not None
                     else np.zeros(space.ndofs))
        self._geom = [element_matrices(space.element_vertices(e), space.p, space.quad, np.eye(3))[0]
                      for e in range(space.nelem)]  # M_e (tissue-free)
        self._dofs = [space.element_dofs(e) for e in range(space.nelem)]

    def _assemble(self, tissue):
        sl, st, th = tissue
        rows, cols, mv, kv = [], [], [], []
        for e in range(self.space.nelem):
            D = diffusion_tensor(sl[e], st[e], th[e])
            _, Ke = element_matrices(self.space.element_vertices(e), self.space.p, self.space.quad, D)
            d = self._dofs[e]
            rows.append(np.repeat(d, d.size))
            cols.append(np.tile(d, d.size))
            mv.append(self._geom[e].reshape(-1))
            kv.append(Ke.reshape(-1))
        r, c = np.concatenate(rows), np.concatenate(cols)
        n = self.space.ndofs
        M = sp.coo_matrix((np.concatenate(mv), (r, c)), shape=(n, n)).tocsr()
        K = sp.coo_matrix((np.concatenate(kv), (r, c)), shape=(n, n)).tocsr()
        return M, K

    def i_app(self, t):
        on = (t > self.t_on) and (t <= self.t_off)
        return self.amplitude * self.mask if on else np.zeros(self.space.ndofs)

    def forward(self, tissue, u0, h0):
        """All states u^0..u^N, h^0..h^N and the traces T[n, s] = u^{n+1}[sensors]."""
        M, K = self._assemble(tissue)
        dt, prm = self.dt, self.prm
        lu1 = spla.splu((M / dt + K).tocsc())
        lu2 = spla.splu((1.5 / dt * M + K).tocsc())
        U = [np.array(u0, dtype=np.float64)]
        H = [np.array(h0, dtype=np.float64)]
        for n in range(self.nsteps):
            t1 = (n + 1) * dt
            if n == 0:
                us = U[0]
                h1 = ionic.gate_bdf1(H[0], us, dt, prm)
                rhs = M @ (U[0] / dt - ionic.i_ion(us, h1, prm) + self.i_app(t1))
                u1 = lu1.solve(rhs)
            else:
                us = 2.0 * U[n] - U[n - 1]
                h1 = ionic.gate_bdf2(H[n], H[n - 1], us, dt, prm)
                rhs = M @ ((4.0 * U[n] - U[n - 1]) / (2.0 * dt) - ionic.i_ion(us, h1, prm) + self.i_app(t1))
                u1 = lu2.solve(rhs)
            U.append(u1)
            H.append(h1)
        traces = np.stack([U[n + 1][self.sensors] for n in range(self.nsteps)])
        return U, H, traces, (M, K, lu1, lu2)

    def gradient(self, tissue, u0, h0, trace_bar):
        """(g_sigma_l, g_sigma_t, g_theta) of a loss with dL/dT = trace_bar."""
        U, H, _, (M, K, lu1, lu2) = self.forward(tissue, u0, h0)
        dt, prm, N = self.dt, self.prm, self.nsteps
        sl, st, th = tissue
        ne = self.space.nelem
        dK = []
        for e in range(ne):
            mats = []
            for dD in _tissue_tensors(sl[e], st[e], th[e]):
                _, Ke = element_matrices(self.space.element_vertices(e), self.space.p, self.space.quad, dD)
                mats.append(Ke)
            dK.append(mats)
        grads = np.zeros((3, ne))
        ubar = [np.zeros(self.space.ndofs) for _ in range(N + 1)]
        hbar = [np.zeros(self.space.ndofs) for _ in range(N + 1)]
        for n in range(N - 1, -1, -1):
            ubar[n + 1][self.sensors] += trace_bar[n]
            w = (lu1 if n == 0 else lu2).solve(ubar[n + 1])
            u1 = U[n + 1]
            for e in range(ne):
                d = self._dofs[e]
                for k in range(3):
                    grads[k, e] -= w[d] @ (dK[e][k] @ u1[d])
            gbar = M @ w
            if n == 0:
                ubar[0] += gbar / dt
                us = U[0]
            else:
                ubar[n] += (2.0 / dt) * gbar
                ubar[n - 1] -= gbar / (2.0 * dt)
                us = 2.0 * U[n] - U[n - 1]
            Ibar = -gbar
            h1 = H[n + 1]
            v = (us - prm["u_rest"]) / prm["u_amp"]
            dI_du = -(h1 * (2.0 * v - 3.0 * v * v) / prm["tau_in"] - 1.0 / prm["tau_out"])
            dI_dh = -prm["u_amp"] * v * v * (1.0 - v) / prm["tau_in"]
            ustar_bar = Ibar * dI_du
            hb = hbar[n + 1] + Ibar * dI_dh
            s = 1.0 / (1.0 + np.exp(-(v - prm["v_gate"]) / prm["kappa"]))
            ds = s * (1.0 - s) / prm["kappa"] / prm["u_amp"]
            a = (1.0 - s) / prm["tau_open"]
            b = s / prm["tau_close"]
            da = -ds / prm["tau_open"]
            db = ds / prm["tau_close"]
            if n == 0:
                D1 = 1.0 + dt * (a + b)
                ustar_bar = ustar_bar + hb * dt * (da - h1 * (da + db)) / D1
                hbar[0] += hb / D1
                ubar[0] += ustar_bar
            else:
                D2 = 3.0 + 2.0 * dt * (a + b)
                ustar_bar = ustar_bar + hb * 2.0 * dt * (da - h1 * (da + db)) / D2
                hbar[n] += 4.0 * hb / D2
                hbar[n - 1] -= hb / D2
                ubar[n] += 2.0 * ustar_bar
                ubar[n - 1] -= ustar_bar
        return grads[0], grads[1], grads[2]


def misfit(traces, target, dt):
    """L = dt/2 sum (T - target)^2 and dL/dT."""
    r = traces - target
    return 0.5 * dt * float(np.sum(r * r)), dt * r
