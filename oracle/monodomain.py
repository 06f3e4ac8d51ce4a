"""Oracle: the partitioned semi-implicit monodomain time step (test infrastructure).

Part of the CPU oracle (plain float64, never called by the product path).

Section 3, Eqs. (ionic_discr), (monodomain_discr), (algebraic_ionic),
(linsys), (matrix_rhs) and Algorithm 1, in the paper's order:

  1. u* = 2 u^n - u^{n-1}                                    (extrapolation)
  2. per DOF: solve the BDF2 gate equation for w^{n+1} at u*,
     then I_ion,i = I_ion(u*_i, w^{n+1}_i)
  3. s = -M I_ion (ionic current interpolation, Eq. algebraic_ionic)
     f = M I_app(x_i, t^{n+1})
     b = M (4 u^n - u^{n-1}) / (2 dt) + s + f                (Eq. matrix_rhs)
  4. solve (3/(2 dt) M + K) u^{n+1} = b                       (Eq. linsys)

Readings of the paper used here:

* First step.  The paper starts at n >= 1 from "suitable initializations"
  of the level-1 values.  This oracle takes one BDF1 step from (u^0, w^0):
  u* = u^0, gate (w^1 - w^0)/dt = H(u^0, w^1),
  (M/dt + K) u^1 = M u^0/dt + s + f.
* Applied current.  The paper writes f_i = I_app(x_i, t^{n+1}); to keep f
  consistent with the ionic term's Galerkin weighting this oracle uses the
  load vector f = M I_app(nodal), i.e. f is to I_app what s is to -I_ion.
* Linear solve.  The exact solution of the sparse SPD system (sparse LU
  direct solve), so the oracle carries no iteration tolerance.
* chi = C_m = 1 as in the paper.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import ionic
from .mesh import SlabSpace, assemble_mass_stiffness


def region_indicator(xyz, region):
    """1.0 where the node lies in the stimulus region, else 0.0.

    region = ("box", (x0, y0, z0, x1, y1, z1)) or ("sphere", (cx, cy, cz, r))."""
    kind, prm = region
    xyz = np.asarray(xyz, dtype=np.float64)
    if kind == "box":
        lo = np.array(prm[:3])
        hi = np.array(prm[3:6])
        inside = np.all((xyz >= lo) & (xyz <= hi), axis=1)
    elif kind == "sphere":
        c = np.array(prm[:3])
        inside = np.sum((xyz - c) ** 2, axis=1) <= prm[3] ** 2
    else:
        raise ValueError(kind)
    return inside.astype(np.float64)


class StandInIonic:
    """The stand-in ionic model of ``oracle.ionic`` with parameters ``prm``."""

    def __init__(self, prm=None):
        self.prm = dict(ionic.DEFAULT_PARAMS if prm is None else prm)

    def gate_first(self, h_n, us, dt):
        return ionic.gate_bdf1(h_n, us, dt, self.prm)

    def gate(self, h_n, h_nm1, us, dt):
        return ionic.gate_bdf2(h_n, h_nm1, us, dt, self.prm)

    def current(self, us, h):
        return ionic.i_ion(us, h, self.prm)


class Monodomain:
    """Assembled-matrix monodomain solver on a slab (Algorithm 2's algebra,
    used as the definition the matrix-free GPU path must reproduce).

    ``model`` supplies the gate update and I_ion (default: the stand-in
    ionic model); ``i_app_fn(t, xyz)``, when given, replaces the region
    stimulus by an arbitrary nodal applied current."""

    def __init__(self, space: SlabSpace, tissue, dt: float, params=None, region=None,
                 amplitude: float = 0.0, t_on: float = 0.0, t_off: float = 0.0,
                 model=None, i_app_fn=None):
        self.space = space
        self.dt = float(dt)
        self.model = StandInIonic(params) if model is None else model
        self.M, self.K = assemble_mass_stiffness(space, tissue)
        self.amplitude, self.t_on, self.t_off = float(amplitude), float(t_on), float(t_off)
        self.i_app_fn = i_app_fn
        self.xyz = space.dof_coordinates() if (region is not None or i_app_fn is not None) else None
        if region is not None:
            self.mask = region_indicator(self.xyz, region)
        else:
            self.mask = np.zeros(space.ndofs)
        self._lu = {}

    def i_app(self, t):
        """Nodal applied current at time t: amplitude on the region for t in (t_on, t_off]."""
        if self.i_app_fn is not None:
            return self.i_app_fn(t, self.xyz)
        on = (t > self.t_on) and (t <= self.t_off)
        return self.amplitude * self.mask if on else np.zeros_like(self.mask)

    def _solve(self, alpha, b):
        if alpha not in self._lu:
            A = (alpha * self.M + self.K).tocsc()
            self._lu[alpha] = spla.splu(A)
        return self._lu[alpha].solve(b)

    def step(self, state):
        """Advance state = dict(u, u_prev, h, h_prev, n) by one time step."""
        dt, model = self.dt, self.model
        u_n, u_nm1, h_n, h_nm1, n = state["u"], state["u_prev"], state["h"], state["h_prev"], state["n"]
        t1 = (n + 1) * dt
        if n == 0:
            us = u_n
            h1 = model.gate_first(h_n, us, dt)
            alpha = 1.0 / dt
            hist = self.M @ (u_n / dt)
        else:
            us = 2.0 * u_n - u_nm1
            h1 = model.gate(h_n, h_nm1, us, dt)
            alpha = 3.0 / (2.0 * dt)
            hist = self.M @ ((4.0 * u_n - u_nm1) / (2.0 * dt))
        s = -(self.M @ model.current(us, h1))
        f = self.M @ self.i_app(t1)
        b = hist + s + f
        u1 = self._solve(alpha, b)
        return dict(u=u1, u_prev=u_n.copy(), h=h1, h_prev=h_n.copy(), n=n + 1)

    def run(self, state, nsteps):
        for _ in range(nsteps):
            state = self.step(state)
        return state


def rest_state(ndofs, prm=None):
    prm = ionic.DEFAULT_PARAMS if prm is None else prm
    u = np.full(ndofs, prm["u_rest"])
    h = np.ones(ndofs)
    return dict(u=u, u_prev=u.copy(), h=h, h_prev=h.copy(), n=0)
