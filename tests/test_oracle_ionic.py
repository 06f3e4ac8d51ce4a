"""Pins of the stand-in ionic model and its BDF gate update (Eq. ionic_discr).

The paper's TTP06 model is not printed, so the ionic model's parity against
the paper is unpinned; what is pinned here is the scheme around it:

* the closed-form BDF1 / BDF2 gate updates solve the implicit BDF equations
  (checked with scipy's bracketing root finder on the residual);
* the single-cell partitioned scheme converges to a fine RK4 solution with
  order 2 in dt;
* rest state: I_ion(u_rest, h) = 0;
* the excitation threshold is the smaller root of the open-gate rate (closed
  form), with return to rest below it and an upstroke above it;
* the gate opens with tau_open below the gate voltage and closes with
  tau_close above it.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import ionic

PRM = ionic.DEFAULT_PARAMS


@pytest.mark.parametrize("u", [-85.0, -72.0, -60.0, -30.0, 10.0])
def test_gate_updates_solve_bdf_equations(u):
    dt = 0.05
    h_n, h_nm1 = 0.7, 0.72

    def res2(h):
        return (3 * h - 4 * h_n + h_nm1) / (2 * dt) - ionic.gate_rhs(u, h, PRM)

    def res1(h):
        return (h - h_n) / dt - ionic.gate_rhs(u, h, PRM)

    h2 = brentq(res2, -1.0, 2.0, xtol=1e-15)
    h1 = brentq(res1, -1.0, 2.0, xtol=1e-15)
    assert abs(float(ionic.gate_bdf2(h_n, h_nm1, u, dt, PRM)) - h2) < 1e-13
    assert abs(float(ionic.gate_bdf1(h_n, u, dt, PRM)) - h1) < 1e-13


def test_rest_state_is_equilibrium_of_the_potential():
    assert abs(float(ionic.i_ion(PRM["u_rest"], 1.0, PRM))) == 0.0


def test_semi_implicit_single_cell_second_order():
    def stim(t):
        return 40.0 * np.exp(-((t - 0.5) / 0.2) ** 2)

    T = 3.0
    ref = ionic.single_cell_rk4(-85.0, 1.0, T, 1e-4, PRM, stim)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        y = ionic.single_cell_semi_implicit(-85.0, 1.0, T, dt, PRM, stim)
        errs.append(abs(y[0] - ref[0]))
    o1 = np.log2(errs[0] / errs[1])
    o2 = np.log2(errs[1] / errs[2])
    assert o1 > 1.7 and o2 > 1.7, errs


def test_action_potential_fires():
    """A supra-threshold start produces an upstroke towards u_rest + u_amp."""
    y = ionic.single_cell_semi_implicit(-60.0, 1.0, 2.0, 0.01, PRM)
    assert y[0] > -10.0


def test_excitation_threshold_is_the_model_root():
    """With the gate open (h = 1) the normalised potential's rate is
    v^2 (1 - v) / tau_in - v / tau_out, which vanishes at the threshold
    v_th = (1 - sqrt(1 - 4 tau_in / tau_out)) / 2 (the smaller nonzero root).
    Starting just below it the cell returns to rest; just above it, it fires."""
    tin, tout = PRM["tau_in"], PRM["tau_out"]
    v_th = 0.5 * (1.0 - np.sqrt(1.0 - 4.0 * tin / tout))
    u_th = PRM["u_rest"] + PRM["u_amp"] * v_th
    assert abs(float(ionic.i_ion(u_th, 1.0, PRM))) < 1e-12 * PRM["u_amp"]
    # near the unstable root the motion is slow: 40 ms to settle, 20 ms to fire
    below = ionic.single_cell_semi_implicit(u_th - 1.0, 1.0, 40.0, 0.01, PRM)
    above = ionic.single_cell_semi_implicit(u_th + 1.0, 1.0, 20.0, 0.01, PRM)
    assert abs(below[0] - PRM["u_rest"]) < 0.5
    assert above[0] > PRM["u_rest"] + 0.7 * PRM["u_amp"]


def test_gate_opens_below_and_closes_above_the_gate_voltage():
    """dh/dt -> (1 - h) / tau_open well below v_gate (the gate opens) and
    -h / tau_close well above it (the gate closes), up to the logistic switch's
    exponentially small overlap."""
    for h in (0.1, 0.6, 0.95):
        low = float(ionic.gate_rhs(PRM["u_rest"], h, PRM))
        high = float(ionic.gate_rhs(PRM["u_rest"] + PRM["u_amp"] * 0.6, h, PRM))
        assert abs(low - (1.0 - h) / PRM["tau_open"]) < 1e-7
        assert abs(high + h / PRM["tau_close"]) < 1e-7
