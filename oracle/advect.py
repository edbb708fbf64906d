"""Semi-Lagrangian advection, explicit viscosity and their adjoints (oracle).

Advection (Sec. 2.3.1, Eq. advection_matrix; Appendix B, Eqs. advection_1 and
advection_2): each face value is the linear (trilinear) interpolation of
``U^n`` at a backtraced point. The two-stage form of Appendix B is read
pointwise as the midpoint rule: from the face position ``x_f``,
``x_m = x_f - dt/2 u(x_f)``, ``x_b = x_f - dt u(x_m)``, ``u~_d = I_d(U^n, x_b)``
where ``u(x)`` interpolates each component on its own staggered lattice.
Sample points are clamped to each lattice's box (periodic grids wrap).

Viscosity (Sec. 2.3.1, Eq. viscosity_matrix; Appendix B, Eq. apply_force):
explicit Euler with the 7-point Laplacian of each component on its own
lattice. Only periodic grids are supported here (the Taylor-Green check).

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


def _laplacian_periodic(u):
    out = -6.0 * u
    for ax in range(3):
        out += np.roll(u, 1, axis=ax) + np.roll(u, -1, axis=ax)
    return out


def viscosity(g: Grid, Ut):
    """``U^ = U~ + nu dt / dx^2 L U~`` (component-wise, periodic grids)."""
    if g.nu == 0.0:
        return [u.copy() for u in Ut]
    if not g.periodic:
        raise NotImplementedError("explicit viscosity is implemented for periodic grids")
    k = g.nu * g.dt / (g.dx * g.dx)
    return [u + k * _laplacian_periodic(u) for u in Ut]


def viscosity_adjoint(g: Grid, gUh):
    """The periodic Laplacian is symmetric, so the adjoint is the same map."""
    return viscosity(g, gUh)
