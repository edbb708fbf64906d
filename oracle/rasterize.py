"""Face fluid fractions and face solid velocities (oracle; tests only).

Sec. 2.3.1 (Projection) introduces alpha^{n+1}, the fluid proportion of each
grid face, computed from the solid's SDF. The reading used here (stated in
the design notes): alpha of a face is the fluid fraction of the dx^3 control
volume centred on that face, estimated with 4 x 4 x 4 cell-centred
subsamples, each contributing a linear ramp ``H(phi) = clamp(1/2 + phi /
(dx / 4), 0, 1)`` one subsample spacing wide, so that alpha is continuous in
the geometry parameters.

The paper's own rule (Sec. 2.3.1, Projection: the zero contour from marching
cubes, its intersections with the face, alpha as the fluid share of the face
area, with the worked single-corner case alpha = 1/2 phi_A/(phi_A - phi_B)
phi_A/(phi_A - phi_D)) is the grid option ``fractions = "corner"``: phi at the
face's four corners, the zero crossing on each edge whose ends differ in
sign placed by linear interpolation, and alpha the area of the polygon
walked around the face through the fluid corners (phi >= 0) and the
crossings, divided by the face area. Where only two diagonal corners are
fluid, that walk keeps the fluid connected across the face (the two solid
corners are cut off).

Box-boundary faces are walls (alpha = 0, u_s = 0) except the outlet patch,
which is open (alpha = 1, Appendix B, Eq. bd:dirichlet), and an optional
inflow patch: wall faces (alpha = 0) whose solid velocity is the prescribed
inflow speed along the wall normal, so the blended update holds them at it
and the right-hand side carries the inflow.
"""

from __future__ import annotations

import itertools

import numpy as np

from . import geometry as geo
from .mac import Grid, boundary_face_mask, face_positions, inlet_face_mask, outlet_face_mask


def subsample_offsets():
    """The 64 subsample offsets in units of dx, (x, y, z) order."""
    pts = []
    for a, b, c in itertools.product(range(4), repeat=3):
        pts.append((np.array([a, b, c], dtype=np.float64) + 0.5) / 4.0 - 0.5)
    return pts


def ramp(phi, dx):
    return np.clip(0.5 + phi / (0.25 * dx), 0.0, 1.0)


def ramp_slope(phi, dx):
    u = 0.5 + phi / (0.25 * dx)
    return np.where((u > 0.0) & (u < 1.0), 4.0 / dx, 0.0)


# corners of a face in cyclic order, in units of dx along its two tangential
# axes (component d's face spans axes (d + 1) % 3 and (d + 2) % 3)
_SQUARE = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])


def corner_polygon(ph):
    """Fluid polygon of the unit square with corner values ``ph`` (4,).

    Returns the vertices and, for each vertex, its derivative with respect to
    the four corner values (a 2 x 4 matrix; zero for a corner vertex).
    """
    verts, dverts = [], []
    for c in range(4):
        n = (c + 1) % 4
        P, Q = _SQUARE[c], _SQUARE[n]
        if ph[c] >= 0.0:
            verts.append(P)
            dverts.append(np.zeros((2, 4)))
        if (ph[c] >= 0.0) != (ph[n] >= 0.0):
            den = ph[c] - ph[n]
            t = ph[c] / den
            verts.append(P + t * (Q - P))
            dt = np.zeros(4)
            dt[c] = -ph[n] / den ** 2
            dt[n] = ph[c] / den ** 2
            dverts.append(np.outer(Q - P, dt))
    return verts, dverts


def corner_fraction(ph):
    """Area of the fluid polygon (the shoelace formula) and its gradient
    with respect to the four corner values."""
    verts, dverts = corner_polygon(np.asarray(ph, dtype=np.float64))
    m = len(verts)
    area, grad = 0.0, np.zeros(4)
    for a in range(m):
        b = (a + 1) % m
        (xa, ya), (xb, yb) = verts[a], verts[b]
        area += 0.5 * (xa * yb - xb * ya)
        grad += 0.5 * (dverts[a][0] * yb + xa * dverts[b][1]
                       - dverts[b][0] * ya - xb * dverts[a][1])
    return area, grad


def face_corners(g: Grid, d):
    """Grid-unit positions ``(..., 4, 3)`` of the corners of component-d faces."""
    X = face_positions(g, d)
    e1, e2 = (d + 1) % 3, (d + 2) % 3
    out = np.repeat(X[..., None, :], 4, axis=-2)
    for c, (s, t) in enumerate(_SQUARE):
        out[..., c, e1] += s - 0.5
        out[..., c, e2] += t - 0.5
    return out


def _corner_fractions(g: Grid, scene, t, d, with_grad):
    K = geo.n_params(scene)
    xc = face_corners(g, d) * g.dx
    ph = geo.phi(scene, xc, t)                          # (..., 4)
    alpha = np.all(ph >= 0.0, axis=-1).astype(np.float64)
    dalpha = np.zeros(alpha.shape + (K,))
    cut = np.argwhere(np.any(ph >= 0.0, axis=-1) & np.any(ph < 0.0, axis=-1))
    dph = geo.dphi_dtheta(scene, xc, t) if (with_grad and K) else None
    for idx in map(tuple, cut):
        a, ga = corner_fraction(ph[idx])
        alpha[idx] = a
        if dph is not None:
            dalpha[idx] = ga @ dph[idx]                 # (4,) @ (4, K)
    return alpha, dalpha


def fractions(g: Grid, scene, t, with_grad=False):
    """alpha per face component (and d alpha / d theta, shape (..., K))."""
    K = geo.n_params(scene)
    if g.fractions == "corner":
        alphas, dalphas = [], []
        for d in range(3):
            alpha, dalpha = _corner_fractions(g, scene, t, d, with_grad)
            wall = boundary_face_mask(g, d)
            alpha[wall] = 0.0
            dalpha[wall] = 0.0
            alpha[outlet_face_mask(g, d)] = 1.0
            alphas.append(alpha)
            dalphas.append(dalpha)
        return (alphas, dalphas) if with_grad else alphas
    alphas, dalphas = [], []
    offs = subsample_offsets()
    for d in range(3):
        xf = face_positions(g, d) * g.dx
        acc = np.zeros(xf.shape[:-1])
        dacc = np.zeros(xf.shape[:-1] + (K,))
        for off in offs:
            xs = xf + off * g.dx
            ph = geo.phi(scene, xs, t)
            acc += ramp(ph, g.dx)
            if with_grad and K:
                dacc += ramp_slope(ph, g.dx)[..., None] * geo.dphi_dtheta(scene, xs, t)
        alpha = acc / 64.0
        dalpha = dacc / 64.0
        wall = boundary_face_mask(g, d)
        alpha[wall] = 0.0
        dalpha[wall] = 0.0
        out = outlet_face_mask(g, d)
        alpha[out] = 1.0
        alphas.append(alpha)
        dalphas.append(dalpha)
    return (alphas, dalphas) if with_grad else alphas


def face_solid_velocity(g: Grid, scene, t, with_grad=False):
    """u_s component d at the centres of component-d faces (0 on the box)."""
    K = geo.n_params(scene)
    us, dus = [], []
    for d in range(3):
        xf = face_positions(g, d) * g.dx
        v = geo.solid_velocity(scene, xf, t)[..., d]
        dv = geo.dus_dtheta(scene, xf, t)[..., d, :] if with_grad else None
        wall = boundary_face_mask(g, d)
        v[wall] = 0.0
        if with_grad:
            dv[wall] = 0.0
        if g.inlet is not None:
            v[inlet_face_mask(g, d)] = float(g.inlet["speed"])
        us.append(v)
        dus.append(dv)
    return (us, dus) if with_grad else us
