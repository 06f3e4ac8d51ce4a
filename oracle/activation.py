"""Oracle: activation times of the transmembrane potential (test infrastructure).

Part of the CPU oracle (plain float64, never called by the product path).

Section 5 (slab results), Eq. (tau): at each node x_i the activation time is
the time at which the approximation of u changes fastest,

    tau(x_i) = argmax_t |du/dt (x_i, t)|,

t running over the discrete time steps and du/dt approximated by the scheme of
the time discretization itself (Section 3): the derivative that belongs to
step n + 1 (time t^{n+1} = (n + 1) dt) is

    BDF1 (first step, n = 0):  (u^1 - u^0) / dt
    BDF2 (n >= 1):             (3 u^{n+1} - 4 u^n + u^{n-1}) / (2 dt).

Readings of the paper used here:

* The derivative of step n + 1 is attached to t^{n+1}, the time of the newest
  value it uses.
* Ties: the earliest step wins (a later step replaces the running maximum only
  when its |du/dt| is strictly larger), so a node that never changes keeps
  tau = t^1.
* Parity unpinned against the paper's printed figures (activation maps of the
  slab and the heart need TTP06 and the paper's geometries); the definition is
  pinned by closed forms (tests/test_oracle_activation.py).
"""
from __future__ import annotations

import numpy as np


def scheme_derivative(u_new, u_cur, u_old, n_new: int, dt: float):
    """du/dt at t^{n_new} by the time scheme: BDF1 for n_new = 1, else BDF2."""
    if n_new == 1:
        return (u_new - u_cur) / dt
    return (3.0 * u_new - 4.0 * u_cur + u_old) / (2.0 * dt)


class ActivationTracker:
    """Running max of |du/dt| per node and the time at which it occurred."""

    def __init__(self, ndofs: int):
        self.dmax = np.full(ndofs, -1.0)
        self.tau = np.full(ndofs, np.nan)

    def update(self, u_new, u_cur, u_old, n_new: int, dt: float):
        d = np.abs(scheme_derivative(u_new, u_cur, u_old, n_new, dt))
        later = d > self.dmax
        self.dmax[later] = d[later]
        self.tau[later] = n_new * dt


def activation_times(history, dt: float):
    """tau and max |du/dt| per node from the states u^0, u^1, ..., u^N (N >= 1)."""
    tr = ActivationTracker(len(history[0]))
    for n_new in range(1, len(history)):
        u_old = history[n_new - 2] if n_new >= 2 else history[0]
        tr.update(history[n_new], history[n_new - 1], u_old, n_new, dt)
    return tr.tau, tr.dmax


def run_with_activation(model, state, nsteps: int):
    """Advance a Monodomain model by nsteps and track activation times on the way;
    returns (final state, tau, max |du/dt|)."""
    tr = ActivationTracker(len(state["u"]))
    for _ in range(nsteps):
        new = model.step(state)
        tr.update(new["u"], state["u"], state["u_prev"], new["n"], model.dt)
        state = new
    return state, tr.tau, tr.dmax
