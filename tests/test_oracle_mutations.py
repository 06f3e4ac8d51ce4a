"""Planted mistakes in the oracle's operator, on the CPU.

Each mutation is a plausible slip in the definition the oracle writes out
(Sections 2-4): a transposed inverse Jacobian, a dropped |det J|, a flipped
fibre angle, a sheet direction that is not orthogonal to the fibre, a
transposed derivative table.  With the mutation in place, at least one pin of
test_oracle_operator must fail; without it, all of them pass.  The test
measures the pins, not the oracle, and leaves the oracle as it found it.
"""
import numpy as np
import pytest

import test_oracle_operator as T
from oracle import element as E
from oracle import mesh as Mh


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
