"""CPU oracle of the matrix-free SEM / SEM-NI monodomain solver (TEST INFRASTRUCTURE).

A plain, slow, float64 restatement of what the paper's method computes,
written from its Sections 2-4 and Algorithms 1-2, sharing no code with the
CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the product package never does.

Modules
  quadrature   LG / LGL rules and the Lagrange basis (Section 3)
  element      dense local mass / stiffness matrices, Eq. (diffusiontensor)
  mesh         slab numbering, assembly (Algorithm 2), element-by-element apply
  ionic        stand-in ionic model and its BDF gate update (parity unpinned
               against the paper: the paper's TTP06 model is not printed)
  monodomain   the partitioned BDF2 time step, Eqs. (ionic_discr)-(matrix_rhs)
"""
from . import element, ionic, mesh, monodomain, quadrature  # noqa: F401
