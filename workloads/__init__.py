"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws and lays out input data: vertex lattices of slab
meshes, per-element tissue parameters and random nodal vectors.  It holds
none of the spectral-element arithmetic (no quadrature, no basis, no
element matrices, no DOF numbering), so that the oracle and the CUDA path
stay independent of each other.

Every generator takes an explicit seed and uses numpy's PCG64 generator.

Workloads (synthetic stand-ins; the Niederer slab benchmark definition and
the Zygote geometries of the paper are not available, so these slabs only
reproduce the shapes and sizes of the paper's workloads):

* ``SLAB_SMALL``   20 x 7 x 3 mm slab, 8 x 4 x 2 hexahedra, affine (no
  perturbation), constant fibre along x.
* ``SLAB_SWEEP``   20 x 7 x 3 mm slab with about 2 million DOFs per degree
  p = 1..6, vertices perturbed by +-10 % of h, fibre angle rotating from
  -60 to +60 degrees through the thickness (z).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Fixed seeds of the synthetic workloads.
SEED_MESH = 1
SEED_U = 2
SEED_STIM = 3
SEED_SENSORS = 4
SEED_SIGMA = 5
SEED_FD = 6

# Slab element counts of the operator-apply sweep: about 2 M DOFs per degree.
SWEEP_ELEMS = {
    1: (333, 116, 50),
    2: (167, 58, 25),
    3: (110, 39, 17),
    4: (83, 29, 13),
    5: (67, 23, 10),
    6: (56, 20, 8),
}

SLAB_LENGTHS_MM = (20.0, 7.0, 3.0)


@dataclass(frozen=True)
class Slab:
    """A structured hexahedral slab: (nx+1)(ny+1)(nz+1) vertices, x fastest."""

    nx: int
    ny: int
    nz: int
    lengths: tuple
    vertices: np.ndarray  # float64 [(nz+1), (ny+1), (nx+1), 3]

    @property
    def n_elements(self) -> int:
        return self.nx * self.ny * self.nz

    def flat_vertices(self) -> np.ndarray:
        """Contiguous float64 array [(nx+1)(ny+1)(nz+1), 3], x fastest."""
        return np.ascontiguousarray(self.vertices.reshape(-1, 3))

    def element_vertices(self) -> np.ndarray:
        """float64 [n_elements, 8, 3]; element order x fastest, corner
        order a + 2 b + 4 c for the corner at (a, b, c) in {0, 1}^3."""
        v = self.vertices
        out = np.empty((self.nz, self.ny, self.nx, 8, 3))
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    out[:, :, :, a + 2 * b + 4 * c, :] = v[c:c + self.nz, b:b + self.ny, a:a + self.nx, :]
        return out.reshape(-1, 8, 3)


def slab(nx: int, ny: int, nz: int, lengths=SLAB_LENGTHS_MM, perturb: float = 0.0,
         seed: int = SEED_MESH) -> Slab:
    """Vertex lattice of a box [0,Lx] x [0,Ly] x [0,Lz] cut into nx*ny*nz hexahedra.

    With ``perturb > 0`` each vertex coordinate is moved by a seeded
    uniform amount in [-perturb*h_d, +perturb*h_d] (h_d the spacing in that
    direction).  A vertex on a face of the box keeps the coordinate normal to
    that face, so the domain stays the same box.
    """
    if min(nx, ny, nz) < 1:
        raise ValueError("a slab needs at least one element per direction")
    lx, ly, lz = (float(x) for x in lengths)
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    zs = np.linspace(0.0, lz, nz + 1)
    v = np.empty((nz + 1, ny + 1, nx + 1, 3))
    v[..., 0] = xs[None, None, :]
    v[..., 1] = ys[None, :, None]
    v[..., 2] = zs[:, None, None]
    if perturb > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        h = np.array([lx / nx, ly / ny, lz / nz])
        d = rng.uniform(-perturb, perturb, size=v.shape) * h
        ix = np.arange(nx + 1)
        iy = np.arange(ny + 1)
        iz = np.arange(nz + 1)
        d[..., 0] *= ((ix > 0) & (ix < nx))[None, None, :]
        d[..., 1] *= ((iy > 0) & (iy < ny))[None, :, None]
        d[..., 2] *= ((iz > 0) & (iz < nz))[:, None, None]
        v = v + d
    return Slab(nx, ny, nz, (lx, ly, lz), v)


def sweep_slab(p: int, seed: int = SEED_MESH) -> Slab:
    """The ~2 M DOF perturbed slab of the operator-apply sweep for degree p."""
    nx, ny, nz = SWEEP_ELEMS[p]
    return slab(nx, ny, nz, SLAB_LENGTHS_MM, perturb=0.1, seed=seed)


def transmural_fiber_angles(s: Slab, theta_min_deg: float = -60.0,
                            theta_max_deg: float = 60.0) -> np.ndarray:
    """Per-element fibre angle (radians) rotating linearly with the
    element-centroid height z / Lz from theta_min to theta_max."""
    zc = s.element_vertices()[:, :, 2].mean(axis=1)
    t = zc / s.lengths[2]
    return np.deg2rad(theta_min_deg + (theta_max_deg - theta_min_deg) * t)


def constant_tissue(s: Slab, sigma_l: float = 0.12, sigma_t: float = 0.03,
                    theta: float = 0.0):
    """Per-element (sigma_l, sigma_t, theta) arrays with constant values."""
    ne = s.n_elements
    return (np.full(ne, float(sigma_l)), np.full(ne, float(sigma_t)), np.full(ne, float(theta)))


def perturbed_conductivities(sigma_l: np.ndarray, sigma_t: np.ndarray, lo: float = 0.8,
                             hi: float = 1.2, seed: int = SEED_SIGMA):
    """Conductivities multiplied by seeded per-element factors in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = rng.uniform(lo, hi, size=(2, sigma_l.size))
    return sigma_l * f[0], sigma_t * f[1]


def uniform_vector(n: int, lo: float = -1.0, hi: float = 1.0, seed: int = SEED_U) -> np.ndarray:
    """Seeded float64 vector with entries uniform in [lo, hi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=int(n))


def seeded_indices(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` distinct seeded indices in [0, n), sorted."""
    rng = np.random.Generator(np.random.PCG64(seed))
    count = min(int(count), int(n))
    return np.sort(rng.choice(int(n), size=count, replace=False))


def seeded_point(lengths, margin: float, seed: int = SEED_STIM) -> np.ndarray:
    """A seeded point inside the box, at least ``margin`` from every face."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.array([rng.uniform(margin, L - margin) for L in lengths])


__all__ = [
    "Slab", "slab", "sweep_slab", "transmural_fiber_angles", "constant_tissue",
    "perturbed_conductivities", "uniform_vector", "seeded_indices", "seeded_point",
    "SWEEP_ELEMS", "SLAB_LENGTHS_MM",
    "SEED_MESH", "SEED_U", "SEED_STIM", "SEED_SENSORS", "SEED_SIGMA", "SEED_FD",
]
