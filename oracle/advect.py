"""Semi-Lagrangian advection, explicit viscosity and their adjoints (oracle).

Advection (Sec. 2.3.1, Eq. advection_matrix; Appendix B, Eqs. advection_1 and
advection_2): each face value is the linear (trilinear) interpolation of
``U^n`` at a backtraced point. The two-stage form of Appendix B is read
pointwise as the midpoint rule: from the face position ``x_f``,
``x_m = x_f - dt/2 u(x_f)``, ``x_b = x_f - dt u(x_m)``, ``u~_d = I_d(U^n, x_b)``
where ``u(x)`` interpolates each component on its own staggered lattice.
Sample points are clamped to each lattice's box (periodic grids wrap).

Viscosity (Sec. 2.3.1, Eq. viscosity_matrix; Appendix B, Eq. apply_force):
explicit Euler ``U^ = (I - nu dt / dx^2 G^T G) U~`` applied to each component
on its own face lattice, where ``G`` takes the difference across every edge
joining two neighbouring lattice points. On a periodic grid the edges wrap
around; in a closed box the lattice ends at the walls and has no edge
beyond them, so ``-G^T G`` is the lattice's graph Laplacian (no flux through
its ends). ``G^T G`` is symmetric, so the adjoint is the same map.

Adjoint (Sec. 2.3.2, Viscosity and Advection): the transpose of the
linearisation, including the dependence of the interpolation weights on the
backtrace positions (the dB/dU U term).
"""

from __future__ import annotations

import numpy as np

from .mac import (Grid, face_positions, trilinear, trilinear_grad,
                  trilinear_scatter, velocity_at)


def _backtrace(g: Grid, U, d, order):
    X = face_positions(g, d)
    v0 = velocity_at(g, U, X)
    if order == 1:
        return X, v0, None, None, X - (g.dt / g.dx) * v0
    Xm = X - (0.5 * g.dt / g.dx) * v0
    v1 = velocity_at(g, U, Xm)
    Xb = X - (g.dt / g.dx) * v1
    return X, v0, Xm, v1, Xb


def advect(g: Grid, U, order=2):
    """``U~ = B(U) U`` for every face component."""
    out = []
    for d in range(3):
        *_, Xb = _backtrace(g, U, d, order)
        out.append(trilinear(g, d, U[d], Xb))
    return out


def advect_adjoint(g: Grid, U, gUt, order=2):
    """``dJ/dU^n`` from ``dJ/dU~`` (weights and positions both differentiated)."""
    gU = [np.zeros_like(u) for u in U]
    for d in range(3):
        X, v0, Xm, v1, Xb = _backtrace(g, U, d, order)
        gval = gUt[d]
        trilinear_scatter(g, d, gU[d], Xb, gval)
        gXb = gval[..., None] * trilinear_grad(g, d, U[d], Xb)
        if order == 1:
            gv0 = -(g.dt / g.dx) * gXb
        else:
            gv1 = -(g.dt / g.dx) * gXb
            gXm = np.zeros_like(Xm)
            for e in range(3):
                trilinear_scatter(g, e, gU[e], Xm, gv1[..., e])
                gXm += gv1[..., e, None] * trilinear_grad(g, e, U[e], Xm)
            gv0 = -(0.5 * g.dt / g.dx) * gXm
        for e in range(3):
            trilinear_scatter(g, e, gU[e], X, gv0[..., e])
    return gU


def _gtg(u, periodic):
    """``G^T G u`` on one component's lattice (array axes = lattice axes)."""
    out = np.zeros_like(u)
    for ax in range(3):
        if periodic:
            e = np.roll(u, -1, axis=ax) - u          # edge (i, i+1), wrapping
            out += np.roll(e, 1, axis=ax) - e        # G^T: +e at i+1, -e at i
        else:
            e = np.diff(u, axis=ax)                  # the n - 1 interior edges
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax] = slice(0, -1)
            hi[ax] = slice(1, None)
            out[tuple(lo)] -= e
            out[tuple(hi)] += e
    return out


def viscosity(g: Grid, Ut):
    """``U^ = (I - nu dt / dx^2 G^T G) U~``, component by component."""
    if g.nu == 0.0:
        return [u.copy() for u in Ut]
    k = g.nu * g.dt / (g.dx * g.dx)
    return [u - k * _gtg(u, g.periodic) for u in Ut]


def viscosity_adjoint(g: Grid, gUh):
    """``G^T G`` is symmetric, so the adjoint is the same map."""
    return viscosity(g, gUh)
