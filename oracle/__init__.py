"""Plain FP64 CPU oracle of the differentiable MAC-grid step.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. It shares no code with the CUDA
path; the two meet only in the seeded inputs of ``nf_inputs``.

What it computes (each module cites the passage it follows):

* ``mac``        MAC grid, unscaled gradient G and its transpose (Sec. 2.3.1).
* ``geometry``   analytic SDF phi, solid velocity u_s and their parameter
                 derivatives for the scenes (Sec. 2.2, Sec. 2.3.3).
* ``rasterize``  face fluid fractions alpha from phi (Sec. 2.3.1, Projection).
* ``advect``     RK2 semi-Lagrangian advection, explicit viscosity and their
                 adjoints (Eqs. advection_matrix, viscosity_matrix; App. B).
* ``project``    cut-cell Poisson system, unpreconditioned CG, velocity
                 update and the projection adjoint (Eqs. projection_matrix,
                 u_next_matrix; Sec. 2.3.2, 2.3.3).
* ``step``       step, rollout, losses, BPTT and central finite differences.
* ``bezier``     polar-Bezier closed curves, their signed distance and radius
                 gradient, extrusion of key cross-sections, CSG (App. A).

Everything is float64 NumPy written for reading, not speed. Every function
is pinned by the ``-m "not gpu"`` tests against results fixed by the
mathematics (symmetry and definiteness of A, dense direct solves, exact
volume fractions of planes, exact shifts, invariants, Taylor-Green decay,
finite differences); see ``tests/test_oracle_*.py``.
"""

from . import advect, bezier, geometry, mac, project, rasterize, step  # noqa: F401
from .mac import Grid  # noqa: F401
