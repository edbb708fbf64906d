"""Face fluid fractions and face solid velocities (oracle; tests only).

Sec. 2.3.1 (Projection) introduces alpha^{n+1}, the fluid proportion of each
grid face, computed from the solid's SDF. The reading used here (stated in
the design notes): alpha of a face is the fluid fraction of the dx^3 control
volume centred on that face, estimated with 4 x 4 x 4 cell-centred
subsamples, each contributing a linear ramp ``H(phi) = clamp(1/2 + phi /
(dx / 4), 0, 1)`` one subsample spacing wide, so that alpha is continuous in
the geometry parameters.

Box-boundary faces are walls (alpha = 0, u_s = 0) except the outlet patch,
which is open (alpha = 1, Appendix B, Eq. bd:dirichlet).
"""

from __future__ import annotations

import itertools

import numpy as np

from . import geometry as geo
from .mac import Grid, boundary_face_mask, face_positions, outlet_face_mask


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


def fractions(g: Grid, scene, t, with_grad=False):
    """alpha per face component (and d alpha / d theta, shape (..., K))."""
    K = geo.n_params(scene)
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
        us.append(v)
        dus.append(dv)
    return (us, dus) if with_grad else us
