"""Pins of the stand-in ionic model and its BDF gate update (Eq. ionic_discr).

The paper's TTP06 model is not printed, so the ionic model's parity against
the paper is unpinned; what is pinned here is the scheme around it:

* the closed-form BDF1 / BDF2 gate updates solve the implicit BDF equations
  (checked with scipy's bracketing root finder on the residual);
* the single-cell partitioned scheme converges to a fine RK4 solution with
  order 2 in dt;
* rest state: I_ion(u_rest, h) = 0.
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
