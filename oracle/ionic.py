"""Oracle: stand-in ionic model and its BDF gate update (test infrastructure).

Part of the CPU oracle (plain float64, never called by the product path).

Section 2, Eq. (monodomain): the ionic model supplies I_ion(u, w, z) and the
gating dynamics dw/dt = H(u, w, z).  The paper uses TTP06 (slab, ventricles)
and CRN (atria) but prints neither model's equations or parameters, so this
build uses a documented two-variable stand-in with the same structure: one
gate h, no concentrations, an I_ion that is nonlinear in u and a gate that
relaxes towards a voltage-dependent target.  Its form is the
Mitchell--Schaeffer model (2003) written in millivolts, with the hard
threshold replaced by a logistic switch so that I_ion and the gate update are
smooth functions of u:

  v      = (u - u_rest) / u_amp                      (normalised potential)
  I_ion  = -u_amp * ( h v^2 (1 - v) / tau_in - v / tau_out )
  s(v)   = 1 / (1 + exp(-(v - v_gate) / kappa))
  dh/dt  = (1 - s) (1 - h) / tau_open  -  s h / tau_close

The parity of this model against the paper is unpinned (the paper's model is
not available); the tests pin it with the exact solution of its linear gate
equation and with a time-convergence check against a fine RK4 reference.

Eq. (ionic_discr): the gate is advanced with BDF2 implicitly in h and with
the extrapolated potential u* = 2u^n - u^{n-1}.  Because dh/dt is affine in h
for fixed u*, the implicit BDF equation is linear in h^{n+1}.
"""
from __future__ import annotations

import numpy as np

DEFAULT_PARAMS = dict(
    u_rest=-85.0,   # mV
    u_amp=100.0,    # mV, upstroke amplitude
    tau_in=0.3,     # ms
    tau_out=6.0,    # ms
    tau_open=120.0,  # ms
    tau_close=150.0,  # ms
    v_gate=0.13,
    kappa=0.01,
)


def normalised(u, prm):
    return (np.asarray(u, dtype=np.float64) - prm["u_rest"]) / prm["u_amp"]


def switch(u, prm):
    v = normalised(u, prm)
    return 1.0 / (1.0 + np.exp(-(v - prm["v_gate"]) / prm["kappa"]))


def i_ion(u, h, prm):
    """Ionic current I_ion(u, h) in mV/ms (chi = C_m = 1)."""
    v = normalised(u, prm)
    return -prm["u_amp"] * (h * v * v * (1.0 - v) / prm["tau_in"] - v / prm["tau_out"])


def gate_rhs(u, h, prm):
    """H(u, h) = dh/dt."""
    s = switch(u, prm)
    return (1.0 - s) * (1.0 - h) / prm["tau_open"] - s * h / prm["tau_close"]


def gate_rates(u, prm):
    """(a, b) with H(u, h) = a (1 - h) - b h."""
    s = switch(u, prm)
    return (1.0 - s) / prm["tau_open"], s / prm["tau_close"]


def gate_bdf2(h_n, h_nm1, u_star, dt, prm):
    """Solve (3 h - 4 h^n + h^{n-1}) / (2 dt) = a(u*) (1 - h) - b(u*) h for h."""
    a, b = gate_rates(u_star, prm)
    return (4.0 * h_n - h_nm1 + 2.0 * dt * a) / (3.0 + 2.0 * dt * (a + b))


def gate_bdf1(h_n, u_star, dt, prm):
    """Solve (h - h^n) / dt = a(u*) (1 - h) - b(u*) h for h (first step)."""
    a, b = gate_rates(u_star, prm)
    return (h_n + dt * a) / (1.0 + dt * (a + b))


def single_cell_rk4(u0, h0, t_end, dt, prm, stim=None):
    """Reference solution of the space-clamped cell du/dt = -I_ion + I_app(t),
    dh/dt = H, by classical RK4 (used only to pin the BDF scheme's order)."""
    def f(t, y):
        u, h = y
        iapp = stim(t) if stim is not None else 0.0
        return np.array([-float(i_ion(u, h, prm)) + iapp, float(gate_rhs(u, h, prm))])

    y = np.array([u0, h0], dtype=np.float64)
    t = 0.0
    nsteps = int(round(t_end / dt))
    for _ in range(nsteps):
        k1 = f(t, y)
        k2 = f(t + dt / 2, y + dt / 2 * k1)
        k3 = f(t + dt / 2, y + dt / 2 * k2)
        k4 = f(t + dt, y + dt * k3)
        y = y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += dt
    return y


def single_cell_semi_implicit(u0, h0, t_end, dt, prm, stim=None):
    """The partitioned scheme of Eqs. (ionic_discr)-(monodomain_discr) on a
    single cell (M = 1, K = 0): BDF1 first step, then BDF2 with u* = 2u^n - u^{n-1}."""
    nsteps = int(round(t_end / dt))
    u_nm1, h_nm1 = u0, h0
    u_n, h_n = u0, h0
    for n in range(nsteps):
        t1 = (n + 1) * dt
        iapp = stim(t1) if stim is not None else 0.0
        if n == 0:
            us = u_n
            h1 = gate_bdf1(h_n, us, dt, prm)
            u1 = u_n + dt * (-float(i_ion(us, h1, prm)) + iapp)
        else:
            us = 2.0 * u_n - u_nm1
            h1 = gate_bdf2(h_n, h_nm1, us, dt, prm)
            u1 = (4.0 * u_n - u_nm1 + 2.0 * dt * (-float(i_ion(us, h1, prm)) + iapp)) / 3.0
        u_nm1, h_nm1, u_n, h_n = u_n, h_n, float(u1), float(h1)
    return np.array([u_n, h_n])

