"""Pins of the activation-time oracle (Eq. tau, Section 5): closed forms of the
BDF1 / BDF2 derivative and brute force on a travelling front."""
import numpy as np
import pytest

from oracle import activation as ACT

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_bdf_derivatives_exact_on_quadratics():
    """BDF2 differentiates quadratics in t exactly, BDF1 linear functions; so on
    u(t) = a t^2 + b t + c the tracked maximum is |2 a t + b| at the step where it
    peaks.  Dyadic dt and coefficients keep every value exact, ties included."""
    dt, nsteps = 1.0 / 16.0, 40
    t = dt * np.arange(nsteps + 1)
    a = np.array([3.0, -2.0, 0.0, 1.0])
    b = np.array([0.5, 1.0, -4.0, -1.5])   # node 3: derivative 2 t - 1.5 vanishes at t = 0.75
    hist = [a * tk ** 2 + b * tk + 1.0 for tk in t]
    d2 = ACT.scheme_derivative(hist[5], hist[4], hist[3], 5, dt)
    assert np.array_equal(d2, 2 * a * t[5] + b)
    # BDF1 of a quadratic at t^1: (u^1 - u^0)/dt = a dt + b
    d1 = ACT.scheme_derivative(hist[1], hist[0], hist[0], 1, dt)
    assert np.array_equal(d1, a * dt + b)
    tau, dmax = ACT.activation_times(hist, dt)
    # nodes 0, 1: |2 a t + b| grows, the last step wins; node 2: constant slope,
    # BDF1 and BDF2 agree exactly, the first step wins (ties keep the earliest)
    assert tau[0] == t[-1] and dmax[0] == abs(2 * a[0] * t[-1] + b[0])
    assert tau[1] == t[-1] and dmax[1] == abs(2 * a[1] * t[-1] + b[1])
    assert tau[2] == t[1] and dmax[2] == 4.0
    # node 3: |2 t - 1.5| is largest at the end (t = 2.5 -> 3.5) against the start
    # (BDF1 at t^1: |dt - 1.5| = 1.4375)
    assert tau[3] == t[-1] and dmax[3] == 3.5


def test_front_arrival_brute_force():
    """A sigmoid upstroke u = tanh((t - t0)/w) per node: the tracked time is the
    step of largest |BDF derivative|, found independently by brute force over the
    sampled derivative, and it lies within one step of t0 (the exact maximum of
    |du/dt|)."""
    rng = np.random.default_rng(3)
    dt, nsteps = 0.05, 200
    t0 = rng.uniform(1.0, 9.0, 64)
    w = rng.uniform(0.2, 0.6, 64)
    t = dt * np.arange(nsteps + 1)
    hist = [np.tanh((tk - t0) / w) for tk in t]
    tau, dmax = ACT.activation_times(hist, dt)
    for i in range(64):
        d = [abs(hist[1][i] - hist[0][i]) / dt] + [
            abs(3 * hist[n][i] - 4 * hist[n - 1][i] + hist[n - 2][i]) / (2 * dt) for n in range(2, nsteps + 1)]
        k = int(np.argmax(d))  # first maximum
        assert tau[i] == pytest.approx(t[k + 1]) and dmax[i] == pytest.approx(d[k])
        assert abs(tau[i] - t0[i]) <= dt + 1e-12


def test_tracker_matches_run_history():
    """Incremental tracking (one update per step) equals the history form."""
    rng = np.random.default_rng(5)
    hist = [rng.standard_normal(30) for _ in range(12)]
    tr = ACT.ActivationTracker(30)
    for n in range(1, 12):
        tr.update(hist[n], hist[n - 1], hist[n - 2] if n >= 2 else hist[0], n, 0.1)
    tau, dmax = ACT.activation_times(hist, 0.1)
    assert np.array_equal(tr.tau, tau) and np.array_equal(tr.dmax, dmax)
