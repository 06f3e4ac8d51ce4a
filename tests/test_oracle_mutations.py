"""Planted mistakes in the oracle, on the CPU.

Each mutation is a plausible slip in a definition the oracle writes out.
- 1-D rules (Section 3): the GLL weight normalisation, Gauss weights without
  their (1 - x^2) factor, a sign slip in the Lagrange derivative.
- Operator (Sections 2-4): a transposed inverse Jacobian, a dropped |det J|,
  a flipped fibre angle, a sheet direction that is not orthogonal to the
  fibre, a transposed derivative table; in the numbering, local i and j
  exchanged, an element's y and z corners exchanged.
- Stand-in ionic model and its gate update (Eq. ionic_discr): a wrong sign of
  the outward current, swapped gate time constants, a wrong sign of the BDF2
  history term.
- Time step (Eqs. monodomain_discr - linsys): the ionic current at u^n
  instead of the extrapolated u*, the BDF1 matrix in BDF2 steps, a wrong sign
  of the history term, an applied current without the mass weighting.
- Multigrid (Section 4.3): a wrong Chebyshev momentum coefficient, one
  post-smoothing step too many, the Lanczos off-diagonal without its square
  root.
- Activation times (Eq. tau): a wrong BDF2 derivative coefficient, ties that
  keep the latest step, the derivative attached to the older time level.
- Adjoint: the conductivity tensor's theta derivative with the wrong sign,
  the sigma_l and sigma_t derivatives swapped.
With the mutation in place at least one pin of the oracle's tests must fail;
without it all of them pass.  The test measures the pins, not the oracle, and
leaves the oracle as it found it.
"""
import warnings

import numpy as np
import pytest

import test_oracle_activation as TA
import test_oracle_adjoint as TAD
import test_oracle_convergence as TC
import test_oracle_ionic as TI
import test_oracle_multigrid as TG
import test_oracle_operator as T
import test_oracle_quadrature as TQ
from oracle import activation as ACT
from oracle import adjoint as AD
from oracle import element as E
from oracle import ionic as I
from oracle import mesh as Mh
from oracle import monodomain as MD
from oracle import multigrid as MG
from oracle import quadrature as Q


def _pins():
    """Runs the operator pins; returns the names of those that fail."""
    checks = [
        ("invariants p=3 LG", lambda: T.test_element_invariants(3, "LG")),
        ("invariants p=3 LGL", lambda: T.test_element_invariants(3, "LGL")),
        ("volume LG", lambda: T.test_volume_on_perturbed_slab("LG", 1)),
        ("exact box p=3 LGL", lambda: T.test_exact_integration_affine_box(3, "LGL")),
        ("exact sheared LG", lambda: T.test_exact_integration_sheared_affine("LG")),
        ("exact sheared LGL", lambda: T.test_exact_integration_sheared_affine("LGL")),
        ("tensor eigenstructure", T.test_diffusion_tensor_eigenstructure),
        ("fibre energy LG", lambda: T.test_linear_field_energy_follows_the_fibre("LG")),
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except (AssertionError, ValueError, np.linalg.LinAlgError):
            failed.append(name)
    return failed


def _matrices(X, p, quad, D, *, transpose_jinv=False, drop_det=False):
    """The oracle's element matrices, with one of two planted geometry slips."""
    phi, dphi, w, pts = E.basis_tables(p, quad)
    _, J = E.trilinear_map(X, pts)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    JinvT = Jinv if transpose_jinv else Jinv.transpose(0, 2, 1)
    Wq = w if drop_det else w * det
    grad = np.einsum("qcd,aqd->aqc", JinvT, dphi)
    return E._mass_stiffness(Wq, phi, grad, D, phi, grad)


_tensor = E.diffusion_tensor


def _tensor_flipped_angle(sl, st, theta, sigma_n=None):
    return _tensor(sl, st, -theta, sigma_n)


def _tensor_bad_sheet(sl, st, theta, sigma_n=None):
    sn = st if sigma_n is None else sigma_n
    f = np.array([np.cos(theta), np.sin(theta), 0.0])
    s = np.array([np.sin(theta), np.cos(theta), 0.0])  # planted: not orthogonal to f
    n = np.array([0.0, 0.0, 1.0])
    return sl * np.outer(f, f) + st * np.outer(s, s) + sn * np.outer(n, n)


_lagrange_deriv = E.lagrange_deriv


def _lagrange_deriv_transposed(nodes, x):
    d = _lagrange_deriv(nodes, x)
    return d.T if d.shape[0] == d.shape[1] else d


MUTATIONS = {
    "inverse Jacobian not transposed": [
        ("element_matrices", lambda X, p, q, D: _matrices(X, p, q, D, transpose_jinv=True))],
    "|det J| dropped": [("element_matrices", lambda X, p, q, D: _matrices(X, p, q, D, drop_det=True))],
    "fibre angle flipped": [("diffusion_tensor", _tensor_flipped_angle)],
    "sheet direction not orthogonal to the fibre": [("diffusion_tensor", _tensor_bad_sheet)],
    "derivative table transposed": [("lagrange_deriv", _lagrange_deriv_transposed)],
}


def _patch(monkeypatch, name, fn):
    for mod in (E, Mh):
        if hasattr(mod, name):
            monkeypatch.setattr(mod, name, fn)


def test_pins_pass_on_the_oracle():
    E.basis_tables.cache_clear()
    assert _pins() == []
    assert _ionic_pins() == []


# ---------------------------------------------------------------- ionic model
def _ionic_pins():
    checks = [("BDF gate u=%g" % u, (lambda u=u: TI.test_gate_updates_solve_bdf_equations(u)))
              for u in (-85.0, -60.0, 10.0)]
    checks += [("rest", TI.test_rest_state_is_equilibrium_of_the_potential),
               ("threshold", TI.test_excitation_threshold_is_the_model_root),
               ("gate direction", TI.test_gate_opens_below_and_closes_above_the_gate_voltage),
               ("fires", TI.test_action_potential_fires)]
    failed = []
    for name, fn in checks:
        try:
            with warnings.catch_warnings(), np.errstate(all="ignore"):
                warnings.simplefilter("ignore")  # a planted mistake may blow the single cell up
                fn()
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(name)
    return failed


_i_ion = I.i_ion
_gate_rates = I.gate_rates


def _i_ion_outward_sign(u, h, prm):  # planted: the outward term with the wrong sign
    v = I.normalised(u, prm)
    return -prm["u_amp"] * (h * v * v * (1.0 - v) / prm["tau_in"] + v / prm["tau_out"])


def _gate_rates_swapped(u, prm):  # planted: opening and closing time constants swapped
    s_ = I.switch(u, prm)
    return (1.0 - s_) / prm["tau_close"], s_ / prm["tau_open"]


def _gate_bdf2_history_sign(h_n, h_nm1, u_star, dt, prm):  # planted: + h^{n-1}
    a, b = _gate_rates(u_star, prm)
    return (4.0 * h_n + h_nm1 + 2.0 * dt * a) / (3.0 + 2.0 * dt * (a + b))


IONIC_MUTATIONS = {
    "outward current sign": ("i_ion", _i_ion_outward_sign),
    "gate time constants swapped": ("gate_rates", _gate_rates_swapped),
    "BDF2 gate history sign": ("gate_bdf2", _gate_bdf2_history_sign),
}


@pytest.mark.parametrize("mutation", sorted(IONIC_MUTATIONS))
def test_each_planted_ionic_mistake_fails_a_pin(mutation, monkeypatch):
    name, fn = IONIC_MUTATIONS[mutation]
    with monkeypatch.context() as m:
        m.setattr(I, name, fn)
        failed = _ionic_pins()
    assert failed, f"no pin caught: {mutation}"


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_each_planted_mistake_fails_a_pin(mutation, monkeypatch):
    E.basis_tables.cache_clear()
    try:
        with monkeypatch.context() as m:
            for name, fn in MUTATIONS[mutation]:
                _patch(m, name, fn)
            failed = _pins()
    finally:
        E.basis_tables.cache_clear()
    assert failed, f"no pin caught: {mutation}"


# ---------------------------------------------------------------- time step


def _step_with(slip):
    """Monodomain.step (Eqs. ionic_discr - linsys) with one planted slip."""
    def step(self, state):
        dt, model = self.dt, self.model
        u_n, u_nm1, h_n, h_nm1, n = state["u"], state["u_prev"], state["h"], state["h_prev"], state["n"]
        t1 = (n + 1) * dt
        if n == 0:
            us = u_n
            h1 = model.gate_first(h_n, us, dt)
            alpha = 1.0 / dt
            hist = self.M @ (u_n / dt)
        else:
            us = u_n if slip == "no extrapolation" else 2.0 * u_n - u_nm1
            h1 = model.gate(h_n, h_nm1, us, dt)
            alpha = 1.0 / dt if slip == "BDF1 matrix in BDF2 steps" else 3.0 / (2.0 * dt)
            sgn = 1.0 if slip == "history sign" else -1.0
            hist = self.M @ ((4.0 * u_n + sgn * u_nm1) / (2.0 * dt))
        s = -(self.M @ model.current(us, h1))
        f = self.i_app(t1) if slip == "unweighted applied current" else self.M @ self.i_app(t1)
        u1 = self._solve(alpha, hist + s + f)
        return dict(u=u1, u_prev=u_n.copy(), h=h1, h_prev=h_n.copy(), n=n + 1)
    return step


STEP_SLIPS = ["no extrapolation", "BDF1 matrix in BDF2 steps", "history sign", "unweighted applied current"]


def _step_pins():
    failed = []
    for name, fn in (("BDF2 order LG", lambda: TC.test_bdf2_time_order("LG")),
                     ("uniform state", TC.test_uniform_state_reduces_to_single_cell)):
        try:
            with warnings.catch_warnings(), np.errstate(all="ignore"):
                warnings.simplefilter("ignore")
                fn()
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(name)
    return failed


def test_step_pins_pass_on_the_oracle(monkeypatch):
    with monkeypatch.context() as m:
        m.setattr(MD.Monodomain, "step", _step_with(None))  # the copy above, unplanted
        assert _step_pins() == []


@pytest.mark.parametrize("slip", STEP_SLIPS)
def test_each_planted_time_step_mistake_fails_a_pin(slip, monkeypatch):
    with monkeypatch.context() as m:
        m.setattr(MD.Monodomain, "step", _step_with(slip))
        failed = _step_pins()
    assert failed, f"no pin caught: {slip}"


# ---------------------------------------------------------------- multigrid

_chebyshev = MG.chebyshev


def _chebyshev_slipped(A, dinv, b, x0, degree, lo, hi):  # planted: rho for rho * rho_old
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = theta / delta
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x if x0 is not None else b.copy()
    d = dinv * r / theta
    x += d
    rho_old = 1.0 / sigma
    for _ in range(1, degree):
        r = b - A @ x
        rho = 1.0 / (2.0 * sigma - rho_old)
        d = rho * d + (2.0 * rho / delta) * (dinv * r)
        x += d
        rho_old = rho
    return x


def _vcycle_post_off_by_one(self, b, level=0):  # planted: one more post-smoothing step
    A, dinv = self.A[level], self.dinv[level]
    lo, hi = self.range[level]
    if level == self.nlevels - 1:
        return _chebyshev(A, dinv, b, None, self.coarse_degree, lo, hi)
    x = _chebyshev(A, dinv, b, None, self.degree, lo, hi)
    r = b - A @ x
    xc = self.vcycle(self.P[level].T @ r, level + 1)
    x = x + self.P[level] @ xc
    return _chebyshev(A, dinv, b, x, self.degree + 1, lo, hi)


def _lanczos_no_sqrt(A, dinv, iters=10):  # planted: beta for sqrt(beta) off the diagonal
    n = A.shape[0]
    r = MG.start_vector(n)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    alphas, betas = [], []
    for _ in range(min(iters, n)):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        r = r - alpha * Ap
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = betas[j] / alphas[j]
    return float(np.linalg.eigvalsh(T).max())


MG_MUTATIONS = {
    "Chebyshev momentum coefficient": (MG, "chebyshev", _chebyshev_slipped),
    "post-smoothing degree off by one": (MG.Hierarchy, "vcycle", _vcycle_post_off_by_one),
    "Lanczos off-diagonal without the square root": (MG, "lanczos_lambda_max", _lanczos_no_sqrt),
}


def _mg_pins():
    failed = []
    for name, fn in (("Chebyshev polynomial", lambda: TG.test_chebyshev_error_polynomial(3)),
                     ("Lanczos bounds", TG.test_lanczos_estimate_bounds_lambda_max),
                     ("V-cycle symmetric, PCG", lambda: TG.test_vcycle_symmetric_and_pcg_converges("LGL"))):
        try:
            with warnings.catch_warnings(), np.errstate(all="ignore"):
                warnings.simplefilter("ignore")
                fn()
        except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError):
            failed.append(name)
    return failed


def test_mg_pins_pass_on_the_oracle():
    assert _mg_pins() == []


@pytest.mark.parametrize("mutation", sorted(MG_MUTATIONS))
def test_each_planted_multigrid_mistake_fails_a_pin(mutation, monkeypatch):
    target, name, fn = MG_MUTATIONS[mutation]
    with monkeypatch.context() as m:
        m.setattr(target, name, fn)
        failed = _mg_pins()
    assert failed, f"no pin caught: {mutation}"


# ---------------------------------------------------------------- activation times

_scheme_derivative = ACT.scheme_derivative


def _derivative_bdf2_coefficient(u_new, u_cur, u_old, n_new, dt):  # planted: 3, -4, +1 -> 3, -4, -1
    if n_new == 1:
        return (u_new - u_cur) / dt
    return (3.0 * u_new - 4.0 * u_cur - u_old) / (2.0 * dt)


def _update_ties_latest(self, u_new, u_cur, u_old, n_new, dt):  # planted: >= keeps the latest tie
    d = np.abs(ACT.scheme_derivative(u_new, u_cur, u_old, n_new, dt))
    later = d >= self.dmax
    self.dmax[later] = d[later]
    self.tau[later] = n_new * dt


def _update_time_of_older_level(self, u_new, u_cur, u_old, n_new, dt):  # planted: t^n for t^{n+1}
    d = np.abs(ACT.scheme_derivative(u_new, u_cur, u_old, n_new, dt))
    later = d > self.dmax
    self.dmax[later] = d[later]
    self.tau[later] = (n_new - 1) * dt


ACT_MUTATIONS = {
    "BDF2 derivative coefficient": (ACT, "scheme_derivative", _derivative_bdf2_coefficient),
    "ties keep the latest step": (ACT.ActivationTracker, "update", _update_ties_latest),
    "derivative attached to the older time": (ACT.ActivationTracker, "update", _update_time_of_older_level),
}


def _act_pins():
    failed = []
    for name, fn in (("quadratics", TA.test_bdf_derivatives_exact_on_quadratics),
                     ("front brute force", TA.test_front_arrival_brute_force)):
        try:
            fn()
        except AssertionError:
            failed.append(name)
    return failed


def test_activation_pins_pass_on_the_oracle():
    assert _act_pins() == []


@pytest.mark.parametrize("mutation", sorted(ACT_MUTATIONS))
def test_each_planted_activation_mistake_fails_a_pin(mutation, monkeypatch):
    target, name, fn = ACT_MUTATIONS[mutation]
    with monkeypatch.context() as m:
        m.setattr(target, name, fn)
        failed = _act_pins()
    assert failed, f"no pin caught: {mutation}"


# ---------------------------------------------------------------- adjoint
_tissue_tensors = AD._tissue_tensors


def _tensors_theta_sign(sl, st, th):  # planted: dD/dtheta with the wrong sign
    ff, rest, dth = _tissue_tensors(sl, st, th)
    return ff, rest, -dth


def _tensors_swapped(sl, st, th):  # planted: dD/dsigma_l and dD/dsigma_t swapped
    ff, rest, dth = _tissue_tensors(sl, st, th)
    return rest, ff, dth


AD_MUTATIONS = {
    "dD/dtheta sign": _tensors_theta_sign,
    "conductivity derivatives swapped": _tensors_swapped,
}


def _ad_pins():
    try:
        TAD.test_adjoint_gradient_matches_central_differences("LGL")
    except AssertionError:
        return ["central differences"]
    return []


def test_adjoint_pins_pass_on_the_oracle():
    assert _ad_pins() == []


@pytest.mark.parametrize("mutation", sorted(AD_MUTATIONS))
def test_each_planted_adjoint_mistake_fails_a_pin(mutation, monkeypatch):
    with monkeypatch.context() as m:
        m.setattr(AD, "_tissue_tensors", AD_MUTATIONS[mutation])
        failed = _ad_pins()
    assert failed, f"no pin caught: {mutation}"


# ---------------------------------------------------------------- quadrature
_gll_rule = Q.gll_rule
_gauss_rule = Q.gauss_rule
_lagrange_deriv_q = Q.lagrange_deriv


def _gll_weights_off(p):  # planted: 2 / (p (p - 1) P_p^2) instead of 2 / (p (p + 1) P_p^2)
    x, w = _gll_rule(p)
    return x, w * (p + 1) / max(p - 1, 1)


def _gauss_weights_no_jacobian(n):  # planted: 2 / P'_n^2, the (1 - x^2) factor dropped
    x, w = _gauss_rule(n)
    return x, w * (1.0 - x * x)


def _lagrange_deriv_wrong_factor(nodes, x):  # planted: one factor of each term inverted
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    dL = np.zeros((n, x.size))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(x.size, 1.0 / (nodes[m] - nodes[i]))
            for l in range(n):
                if l != i and l != m:
                    term *= (x - nodes[l]) / (nodes[i] - nodes[l])
            dL[i] += term
    return dL


Q_MUTATIONS = {
    "GLL weight normalisation": ("gll_rule", _gll_weights_off),
    "Gauss weights without 1 - x^2": ("gauss_rule", _gauss_weights_no_jacobian),
    "Lagrange derivative sign": ("lagrange_deriv", _lagrange_deriv_wrong_factor),
}


def _q_pins():
    checks = [("GLL textbook", TQ.test_gll_textbook_values),
              ("Gauss textbook", TQ.test_gauss_textbook_values),
              ("derivative vs polyfit", TQ.test_lagrange_derivative_matches_numpy_polyfit)]
    checks += [("LG exact p=%d" % p, (lambda p=p: TQ.test_lg_exactness_degree(p))) for p in (2, 4)]
    checks += [("LGL exact p=%d" % p, (lambda p=p: TQ.test_lgl_exactness_degree(p))) for p in (2, 4)]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except AssertionError:
            failed.append(name)
    return failed


def test_quadrature_pins_pass_on_the_oracle():
    assert _q_pins() == []


@pytest.mark.parametrize("mutation", sorted(Q_MUTATIONS))
def test_each_planted_quadrature_mistake_fails_a_pin(mutation, monkeypatch):
    name, fn = Q_MUTATIONS[mutation]
    with monkeypatch.context() as m:
        m.setattr(Q, name, fn)
        failed = _q_pins()
    assert failed, f"no pin caught: {mutation}"


# ---------------------------------------------------------------- numbering
_element_dofs = Mh.SlabSpace.element_dofs


def _element_dofs_i_j_swapped(self, e):  # planted: local i and j exchanged
    ex, ey, ez = self.element_ijk(e)
    n, p = self.n, self.p
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    g = (ex * p + j) + self.NX * ((ey * p + i) + self.NY * (ez * p + k))
    return g.reshape(-1)


def _element_vertices_b_c_swapped(self, e):  # planted: the y and z corners exchanged
    ex, ey, ez = self.element_ijk(e)
    X = np.empty((8, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                X[a + 2 * b + 4 * c] = self.V[ez + b, ey + c, ex + a]
    return X


NUMBERING_MUTATIONS = {
    "local i and j exchanged": ("element_dofs", _element_dofs_i_j_swapped),
    "element corners y and z exchanged": ("element_vertices", _element_vertices_b_c_swapped),
}


@pytest.mark.parametrize("mutation", sorted(NUMBERING_MUTATIONS))
def test_each_planted_numbering_mistake_fails_a_pin(mutation, monkeypatch):
    name, fn = NUMBERING_MUTATIONS[mutation]
    E.basis_tables.cache_clear()
    with monkeypatch.context() as m:
        m.setattr(Mh.SlabSpace, name, fn)
        failed = _pins()
    assert failed, f"no pin caught: {mutation}"
