"""The seeded input recipe (workloads/): the shapes and structure the tests and
the bench rely on.  No method arithmetic lives there; these checks pin the
recipe itself."""
import numpy as np

import workloads as W


def test_perturbed_slab_keeps_the_box():
    s = W.slab(6, 4, 3, (20.0, 7.0, 3.0), perturb=0.1, seed=1)
    v = s.flat_vertices().reshape(s.nz + 1, s.ny + 1, s.nx + 1, 3)
    h = np.array([20.0 / 6, 7.0 / 4, 3.0 / 3])
    base = W.slab(6, 4, 3, (20.0, 7.0, 3.0)).flat_vertices().reshape(v.shape)
    d = v - base
    assert np.all(np.abs(d) <= 0.1 * h + 1e-12)
    # a vertex on a face keeps the coordinate normal to it
    assert np.all(d[:, :, 0, 0] == 0) and np.all(d[:, :, -1, 0] == 0)
    assert np.all(d[:, 0, :, 1] == 0) and np.all(d[:, -1, :, 1] == 0)
    assert np.all(d[0, :, :, 2] == 0) and np.all(d[-1, :, :, 2] == 0)
    # and the interior moves
    assert np.abs(d[1:-1, 1:-1, 1:-1]).max() > 0.05 * h.min()


def test_seeded_inputs_are_reproducible():
    a = W.slab(5, 3, 2, perturb=0.1, seed=7).flat_vertices()
    b = W.slab(5, 3, 2, perturb=0.1, seed=7).flat_vertices()
    c = W.slab(5, 3, 2, perturb=0.1, seed=8).flat_vertices()
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(W.uniform_vector(100, seed=2), W.uniform_vector(100, seed=2))


def test_sweep_slabs_hold_about_two_million_dofs():
    for p in range(1, 7):
        s = W.sweep_slab(p)
        ndofs = (p * s.nx + 1) * (p * s.ny + 1) * (p * s.nz + 1)
        assert 1.9e6 < ndofs < 2.1e6, (p, ndofs)
    s4 = W.sweep_slab(4)
    assert (s4.nx, s4.ny, s4.nz) == (83, 29, 13)


def test_transmural_fibres_rotate_from_minus_to_plus_sixty_degrees():
    s = W.slab(4, 3, 10, (20.0, 7.0, 3.0))
    th = W.transmural_fiber_angles(s)
    assert th.shape == (s.n_elements,)
    assert np.all(th >= np.radians(-60.0) - 1e-15) and np.all(th <= np.radians(60.0) + 1e-15)
    # constant within a z-layer, increasing with z
    layers = th.reshape(s.nz, s.ny * s.nx)
    assert np.all(layers.max(axis=1) == layers.min(axis=1))
    assert np.all(np.diff(layers[:, 0]) > 0)
