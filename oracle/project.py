"""Cut-cell pressure projection and its adjoint (FP64 oracle; tests only).

Sec. 2.3.1 (Projection), Eq. projection_matrix: with ``S = diag(alpha)`` and
``c = dt / (rho dx)``,

    A P = b,   A = c G^T S G,   b = G^T S U^ + G^T (I - S) U_s,

solved here by *unpreconditioned* conjugate gradients from ``P = 0`` until
``||b - A P|| / ||b|| <= tol`` (a plain definition of the same solution the
multigrid-preconditioned solver reaches).

Velocity update (Eq. u_next_matrix), in the blended reading used throughout:
``U = S (U^ - c G P) + (I - S) U_s``: equal to the paper's update on fluid
faces (alpha = 1), to the solid velocity on solid faces (alpha = 0, Eq.
bd:neumann), and continuous in alpha in between. ``velocity_rule="literal"``
gives the paper's printed update ``U^ - c G P`` for comparison.

Active cells: a cell takes part iff the sum of its six face fractions is
positive; other cells keep ``P = 0``. Connected fluid components (cells
linked through faces with alpha > 0) that touch no open boundary face have a
constant null space; there the right-hand side is projected to zero mean (a
no-op for consistent data) and the pressure is fixed to zero mean.

Adjoint (Sec. 2.3.2, Projection; Sec. 2.3.3), written as the exact transpose
of the forward above with ``A y = dJ/dP`` (A is symmetric):

    gS   = gU (U^ - c G P - U_s) + (G y)(U^ - U_s) - c (G y)(G P)
    gU^  = S (gU + G y),    gU_s = (I - S)(gU + G y),   gP = -c G^T S gU.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from .mac import Grid, axis_of, grad, grad_T


class NotConverged(RuntimeError):
    pass


def face_sum(g: Grid, alpha):
    """Sum of the six face fractions around each cell."""
    s = np.zeros(g.cell_shape)
    for d in range(3):
        ax = axis_of(d)
        a = alpha[d]
        if g.periodic:
            s += a + np.roll(a, -1, axis=ax)
        else:
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax] = slice(0, -1)
            hi[ax] = slice(1, None)
            s += a[tuple(lo)] + a[tuple(hi)]
    return s


def active_cells(g: Grid, alpha):
    return face_sum(g, alpha) > 0.0


def components(g: Grid, alpha, active):
    """Labels of fluid components and whether each touches an open face.

    Returns ``(labels, grounded)``: ``labels`` is -1 on inactive cells.
    """
    shp = g.cell_shape
    ncell = int(np.prod(shp))
    lin = np.arange(ncell).reshape(shp)
    rows, cols = [], []
    for d in range(3):
        ax = axis_of(d)
        a = alpha[d]
        if g.periodic:
            left = lin
            right = np.roll(lin, -1, axis=ax)
            af = np.roll(a, -1, axis=ax)       # face between cell and +1 cell
        else:
            sl = [slice(None)] * 3
            sl[ax] = slice(1, -1)
            af = a[tuple(sl)]
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax] = slice(0, -1)
            hi[ax] = slice(1, None)
            left, right = lin[tuple(lo)], lin[tuple(hi)]
        m = af > 0.0
        rows.append(left[m])
        cols.append(right[m])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    adj = sp.coo_matrix((np.ones(len(r)), (r, c)), shape=(ncell, ncell))
    _, lab = connected_components(adj, directed=False)
    lab = lab.reshape(shp)
    labels = np.where(active, lab, -1)
    grounded = {}
    # open boundary faces: boundary faces with alpha > 0
    touch = np.zeros(shp, dtype=bool)
    if not g.periodic:
        for d in range(3):
            ax = axis_of(d)
            a = alpha[d]
            first = [slice(None)] * 3
            last = [slice(None)] * 3
            first[ax] = 0
            last[ax] = -1
            cfirst = [slice(None)] * 3
            clast = [slice(None)] * 3
            cfirst[ax] = 0
            clast[ax] = -1
            t0 = np.zeros(shp, dtype=bool)
            t0[tuple(cfirst)] = a[tuple(first)] > 0.0
            t1 = np.zeros(shp, dtype=bool)
            t1[tuple(clast)] = a[tuple(last)] > 0.0
            touch |= t0 | t1
    for lab_id in np.unique(labels[labels >= 0]):
        grounded[int(lab_id)] = bool(np.any(touch[labels == lab_id]))
    return labels, grounded


def remove_floating_means(v, labels, grounded):
    """Zero the mean of ``v`` on every component without an open face."""
    v = v.copy()
    for lab_id, gr in grounded.items():
        if not gr:
            m = labels == lab_id
            v[m] -= v[m].mean()
    return v


def apply_A(g: Grid, alpha, active, p):
    """``A p = c G^T S G p`` restricted to active cells."""
    pa = np.where(active, p, 0.0)
    Gp = grad(g, pa)
    return np.where(active, g.c * grad_T(g, [alpha[d] * Gp[d] for d in range(3)]), 0.0)


def cg(apply, b, tol, max_iter=100000):
    """Unpreconditioned CG from x = 0; stops on the true relative residual."""
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    r = b.copy()
    d = r.copy()
    rr = float(np.vdot(r, r))
    it = 0
    while it < max_iter:
        q = apply(d)
        dq = float(np.vdot(d, q))
        if dq <= 0.0:
            break
        a = rr / dq
        x += a * d
        r -= a * q
        rr_new = float(np.vdot(r, r))
        it += 1
        if np.sqrt(rr_new) / bn <= tol:
            rt = b - apply(x)
            rel = np.linalg.norm(rt) / bn
            if rel <= tol:
                return x, it, rel
            r = rt                       # restart from the true residual
            rr_new = float(np.vdot(r, r))
            d = r.copy()
            rr = rr_new
            continue
        d = r + (rr_new / rr) * d
        rr = rr_new
    rel = np.linalg.norm(b - apply(x)) / bn
    if rel <= tol:
        return x, it, rel
    raise NotConverged(f"CG stopped at {it} iterations, relative residual {rel:.3e}")


class ProjectionSystem:
    """The linear system of one projection: alpha, u_s, active set, gauge."""

    def __init__(self, g: Grid, alpha, us):
        self.g = g
        self.alpha = alpha
        self.us = us
        self.active = active_cells(g, alpha)
        self.labels, self.grounded = components(g, alpha, self.active)

    def A(self, p):
        return apply_A(self.g, self.alpha, self.active, p)

    def solve(self, rhs, tol):
        rhs = np.where(self.active, rhs, 0.0)
        rhs = remove_floating_means(rhs, self.labels, self.grounded)
        x, it, rel = cg(self.A, rhs, tol)
        x = remove_floating_means(np.where(self.active, x, 0.0), self.labels, self.grounded)
        return x, it, rel

    def rhs(self, Uh):
        a, us = self.alpha, self.us
        return np.where(self.active,
                        grad_T(self.g, [a[d] * Uh[d] + (1.0 - a[d]) * us[d] for d in range(3)]),
                        0.0)


def project(g: Grid, alpha, us, Uh, tol, velocity_rule="blend"):
    """Solve Eq. projection_matrix and apply the velocity update."""
    sys_ = ProjectionSystem(g, alpha, us)
    b = sys_.rhs(Uh)
    P, it, rel = sys_.solve(b, tol)
    GP = grad(g, P)
    if velocity_rule == "blend":
        U = [alpha[d] * (Uh[d] - g.c * GP[d]) + (1.0 - alpha[d]) * us[d] for d in range(3)]
    elif velocity_rule == "literal":
        U = [Uh[d] - g.c * GP[d] for d in range(3)]
    else:
        raise ValueError(velocity_rule)
    info = dict(iters=it, rel_residual=rel, system=sys_, b=b)
    return U, P, info


def project_adjoint(g: Grid, alpha, us, Uh, P, gU, tol, system=None):
    """Transpose of :func:`project` (blended rule).

    Returns ``(gUh, gS, gUs, y, info)`` with ``gS`` and ``gUs`` per face.
    """
    sys_ = system if system is not None else ProjectionSystem(g, alpha, us)
    c = g.c
    GP = grad(g, P)
    gS = [gU[d] * (Uh[d] - c * GP[d] - us[d]) for d in range(3)]
    gP = -c * grad_T(g, [alpha[d] * gU[d] for d in range(3)])
    y, it, rel = sys_.solve(gP, tol)
    Gy = grad(g, y)
    gUh = [alpha[d] * (gU[d] + Gy[d]) for d in range(3)]
    gUs = [(1.0 - alpha[d]) * (gU[d] + Gy[d]) for d in range(3)]
    for d in range(3):
        gS[d] = gS[d] + Gy[d] * (Uh[d] - us[d]) - c * Gy[d] * GP[d]
    return gUh, gS, gUs, y, dict(iters=it, rel_residual=rel)
