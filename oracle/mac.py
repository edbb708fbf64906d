"""MAC grid operators of the FP64 oracle (test infrastructure only).

Sec. 2.3.1 (Numerical Simulation): pressures live at cell centres, velocity
components on the faces normal to them; ``G / dx`` is the gradient and
``-G^T / dx`` the divergence. ``G`` here is the unscaled +-1 face difference.
Outside the box the ghost pressure is zero (Appendix B, Eq. bd:dirichlet);
whether a boundary face then acts as a wall or as an open face is decided by
its fluid fraction (0 on walls, 1 on the outlet).

Positions are handled in grid units ``X = x / dx``. The face of component
``d`` with array index ``(k, j, i)`` sits at ``X = (i, j, k) + 1/2`` except
along axis ``d`` where the half is absent. Component ``e``'s samples form the
lattice ``X - shift_e`` with ``shift_e = 1/2`` on every axis but ``e``.
"""

from __future__ import annotations

import copy

import numpy as np


class Grid:
    """Plain description of the grid and time step (``c = dt / (rho dx)``)."""

    def __init__(self, desc):
        self.nx, self.ny, self.nz = desc["nx"], desc["ny"], desc["nz"]
        self.dx = float(desc["dx"])
        self.dt = float(desc["dt"])
        self.rho = float(desc.get("rho", 1.0))
        self.nu = float(desc.get("nu", 0.0))
        self.periodic = bool(desc.get("periodic", False))
        # face fractions: "supersample" (4x4x4 ramp samples of the face's
        # control volume) or "corner" (face area from the corner values)
        self.fractions = desc.get("fractions", "supersample")
        if self.fractions not in ("supersample", "corner"):
            raise ValueError(f"unknown fraction rule {self.fractions!r}")
        self.outlet = desc.get("outlet")
        # an inflow patch: boundary faces held at a prescribed normal velocity
        # (a wall, alpha = 0, whose solid velocity is the inflow)
        self.inlet = desc.get("inlet")
        self.c = self.dt / (self.rho * self.dx)
        self.n = (self.nx, self.ny, self.nz)          # cells per axis, (x, y, z)

    @property
    def cell_shape(self):
        return (self.nz, self.ny, self.nx)

    def face_shape(self, d):
        if self.periodic:
            return self.cell_shape
        s = list(self.cell_shape)
        s[2 - d] += 1
        return tuple(s)

    def zeros_faces(self):
        return [np.zeros(self.face_shape(d)) for d in range(3)]

    def with_dt(self, h):
        """The same grid for a step of length h (advection and c = h / (rho dx))."""
        g = copy.copy(self)
        g.dt = float(h)
        g.c = g.dt / (g.rho * g.dx)
        return g


def axis_of(d):
    """Array axis holding spatial axis ``d`` (arrays are indexed [z, y, x])."""
    return 2 - d


def grad(g: Grid, P):
    """Unscaled MAC gradient ``G P`` (one value per face, ghost pressure 0)."""
    out = []
    for d in range(3):
        ax = axis_of(d)
        if g.periodic:
            out.append(P - np.roll(P, 1, axis=ax))
        else:
            pad = [(0, 0)] * 3
            pad[ax] = (1, 1)
            out.append(np.diff(np.pad(P, pad), axis=ax))
    return out


def grad_T(g: Grid, V):
    """Exact transpose ``G^T V`` (equals ``-dx * divergence``)."""
    out = np.zeros(g.cell_shape)
    for d in range(3):
        ax = axis_of(d)
        if g.periodic:
            out += V[d] - np.roll(V[d], -1, axis=ax)
        else:
            out -= np.diff(V[d], axis=ax)
    return out


def face_positions(g: Grid, d):
    """Grid-unit positions ``(..., 3)`` (x, y, z order) of component-d faces."""
    shp = g.face_shape(d)
    k, j, i = np.meshgrid(np.arange(shp[0]), np.arange(shp[1]),
                          np.arange(shp[2]), indexing="ij")
    X = np.stack([i, j, k], axis=-1).astype(np.float64) + 0.5
    X[..., d] -= 0.5
    return X


def boundary_face_mask(g: Grid, d):
    """True on faces of component d lying on the box boundary."""
    m = np.zeros(g.face_shape(d), dtype=bool)
    if g.periodic:
        return m
    ax = axis_of(d)
    idx = [slice(None)] * 3
    idx[ax] = 0
    m[tuple(idx)] = True
    idx[ax] = -1
    m[tuple(idx)] = True
    return m


def inlet_face_mask(g: Grid, d):
    """True on the boundary faces of the inflow patch (an x wall)."""
    m = np.zeros(g.face_shape(d), dtype=bool)
    o = g.inlet
    if o is None or g.periodic or d != o["axis"]:
        return m
    assert o["axis"] == 0, "inflow patches are on an x wall"
    i = g.nx if o["side"] > 0 else 0
    m[o["k0"]:o["k0"] + o["h"], o["j0"]:o["j0"] + o["w"], i] = True
    return m


def outlet_face_mask(g: Grid, d):
    """True on the boundary faces forming the open outlet patch."""
    m = np.zeros(g.face_shape(d), dtype=bool)
    o = g.outlet
    if o is None or g.periodic or d != o["axis"]:
        return m
    assert o["axis"] == 0, "outlet patches are on an x wall"
    i = g.nx if o["side"] > 0 else 0
    m[o["k0"]:o["k0"] + o["h"], o["j0"]:o["j0"] + o["w"], i] = True
    return m


# ------------------------------------------------------- interpolation ----

def _axis_weights(gpos, npts, periodic):
    """Split lattice coordinates into cell index, fraction and clamp slope.

    Non-periodic: the coordinate is clamped to ``[0, npts - 1]`` (the sample
    box of this lattice); the returned ``slope`` is the derivative of the
    clamp (1 inside the closed box, 0 outside).
    """
    if periodic:
        gw = np.mod(gpos, npts)
        i0 = np.floor(gw).astype(np.int64)
        f = gw - i0
        i0 = np.mod(i0, npts)
        i1 = np.mod(i0 + 1, npts)
        slope = np.ones_like(gpos)
    else:
        L = npts - 1
        slope = ((gpos >= 0.0) & (gpos <= L)).astype(np.float64)
        gc = np.clip(gpos, 0.0, float(L))
        i0 = np.clip(np.floor(gc).astype(np.int64), 0, L - 1)
        f = gc - i0
        i1 = i0 + 1
    return i0, i1, f, slope


def lattice_points(g: Grid, e):
    """Sample count per axis (x, y, z) of component e's lattice."""
    n = list(g.n)
    if not g.periodic:
        n[e] += 1
    return n


def trilinear_stencil(g: Grid, e, X):
    """Corners and weights of the trilinear interpolant of component ``e``.

    Returns ``(corners, dweights)`` where ``corners`` is a list of 8
    ``(index tuple, weight)`` and ``dweights[a]`` the list of the 8 weights'
    derivatives with respect to the grid-unit position along axis ``a``.
    """
    npts = lattice_points(g, e)
    shift = np.full(3, 0.5)
    shift[e] = 0.0
    ax = [_axis_weights(X[..., a] - shift[a], npts[a], g.periodic)
          for a in range(3)]
    corners = []
    dweights = [[], [], []]
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                c = (cx, cy, cz)
                idx = []
                w = np.ones(X.shape[:-1])
                per_axis = []
                for a in range(3):
                    i0, i1, f, _ = ax[a]
                    idx.append(i1 if c[a] else i0)
                    wa = f if c[a] else 1.0 - f
                    per_axis.append(wa)
                    w = w * wa
                corners.append(((idx[2], idx[1], idx[0]), w))
                for a in range(3):
                    slope = ax[a][3]
                    dwa = slope * (1.0 if c[a] else -1.0)
                    others = np.ones(X.shape[:-1])
                    for b in range(3):
                        if b != a:
                            others = others * per_axis[b]
                    dweights[a].append(dwa * others)
    return corners, dweights


def trilinear(g: Grid, e, Ue, X):
    """Value of component ``e``'s trilinear interpolant at positions X."""
    corners, _ = trilinear_stencil(g, e, X)
    out = np.zeros(X.shape[:-1])
    for idx, w in corners:
        out += w * Ue[idx]
    return out


def trilinear_grad(g: Grid, e, Ue, X):
    """Gradient (grid units) of component e's interpolant at X, ``(..., 3)``."""
    corners, dw = trilinear_stencil(g, e, X)
    out = np.zeros(X.shape)
    for a in range(3):
        for (idx, _), dwa in zip(corners, dw[a]):
            out[..., a] += dwa * Ue[idx]
    return out


def trilinear_scatter(g: Grid, e, target, X, gval):
    """Adjoint of :func:`trilinear` w.r.t. the samples: target += W^T gval."""
    corners, _ = trilinear_stencil(g, e, X)
    for idx, w in corners:
        np.add.at(target, idx, w * gval)


def velocity_at(g: Grid, U, X):
    """The three interpolated components at positions X, ``(..., 3)``."""
    return np.stack([trilinear(g, e, U[e], X) for e in range(3)], axis=-1)
