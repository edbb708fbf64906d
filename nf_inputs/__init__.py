"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds grid and scene *descriptions* and seeded random draws only.
No step of the method's arithmetic (geometry evaluation, rasterisation,
advection, projection, adjoint) lives here, so the oracle and the CUDA path
can both consume these inputs without sharing any solver code.

Conventions of the descriptions (both consumers follow them):

* Unit-spaced MAC grid of ``nx * ny * nz`` cells with spacing ``dx``. Face
  arrays are stored per component with x fastest: ``u[0]`` has shape
  ``(nz, ny, nx + 1)``, ``u[1]`` ``(nz, ny + 1, nx)``, ``u[2]``
  ``(nz + 1, ny, nx)``; cell arrays have shape ``(nz, ny, nx)``. A periodic
  grid (oracle only) stores ``(nz, ny, nx)`` for every component.
* ``outlet`` is ``None`` or a dict ``{"axis": 0, "side": 1, "j0", "k0", "w",
  "h"}``: the patch of boundary faces on the high-x wall whose y-cell index is
  in ``[j0, j0 + w)`` and z-cell index in ``[k0, k0 + h)``.
* A scene is ``{"kind": ..., "theta": [...], **constants}`` with kinds
  ``none``, ``sphere``, ``chamber``, ``plate`` and ``spheres``; ``theta`` holds
  the differentiable parameters (design and control).
"""

from __future__ import annotations

import numpy as np

SCENE_KINDS = ("none", "sphere", "chamber", "plate", "spheres", "shell")


def make_grid(n, dt, *, ny=None, nz=None, nu=0.0, rho=1.0, outlet=None,
              periodic=False, extent=1.0, inlet=None):
    """A grid description: ``n`` cells along x over ``[0, extent]``."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    g = dict(nx=int(n), ny=int(ny), nz=int(nz), dx=float(extent) / n,
             dt=float(dt), rho=float(rho), nu=float(nu),
             periodic=bool(periodic), outlet=outlet)
    if inlet is not None:
        g["inlet"] = inlet
    return g


def face_shape(grid, d):
    """Array shape of face component ``d`` (0 = x, 1 = y, 2 = z)."""
    nx, ny, nz = grid["nx"], grid["ny"], grid["nz"]
    if grid.get("periodic", False):
        return (nz, ny, nx)
    return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][d]


def cell_shape(grid):
    return (grid["nz"], grid["ny"], grid["nx"])


def centred_outlet(n, width):
    """A ``width x width`` patch of high-x boundary faces centred in (y, z)."""
    j0 = n // 2 - width // 2
    return dict(axis=0, side=1, j0=j0, k0=j0, w=int(width), h=int(width))


def centred_inlet(n, width, speed, side=-1):
    """A ``width x width`` inflow patch of x-wall faces centred in (y, z),
    holding the normal velocity ``speed`` (along +x on the low-x wall)."""
    j0 = n // 2 - width // 2
    return dict(axis=0, side=int(side), j0=j0, k0=j0, w=int(width), h=int(width),
                speed=float(speed))


def gaussian_faces(grid, sigma, seed):
    """Independent N(0, sigma^2) values on every face (PCG64 with ``seed``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [sigma * rng.standard_normal(face_shape(grid, d)) for d in range(3)]


def zero_faces(grid):
    return [np.zeros(face_shape(grid, d)) for d in range(3)]


# ---------------------------------------------------------------- scenes ----

def sphere_scene(v=(0.1, 0.0, 0.0), centre=(0.5, 0.5, 0.5), radius=0.2):
    """A solid sphere translating with constant velocity ``theta = v``."""
    return dict(kind="sphere", theta=[float(x) for x in v],
                centre=[float(x) for x in centre], radius=float(radius))


def chamber_scene(theta, dx, *, centre=(0.5, 0.5, 0.5),
                  axes=(0.35, 0.25, 0.25), period=0.5, duct_x0=0.5,
                  duct_half_cells=8):
    """Pulsing ellipsoidal chamber joined to an outlet duct.

    ``theta = (a1..a4, b1..b4)`` are the Fourier coefficients of the radius
    modulation. The duct is the slab ``x >= duct_x0`` with square cross
    section of half width ``duct_half_cells * dx`` centred at (0.5, 0.5).
    """
    theta = [float(x) for x in theta]
    assert len(theta) == 8
    return dict(kind="chamber", theta=theta, centre=[float(x) for x in centre],
                axes=[float(x) for x in axes], period=float(period),
                duct_x0=float(duct_x0), duct_half=float(duct_half_cells * dx))


def plate_scene(theta, dx, period, *, centre=(0.5, 0.5, 0.5),
                half=(0.3, None, 0.3)):
    """Flat plate hinged at ``centre`` rotating about z.

    ``theta`` holds 4 angle knots at t = 0, T/3, 2T/3, T (T = ``period``); the
    plate is 3 cells thick (half thickness 1.5 dx) unless ``half`` says
    otherwise.
    """
    theta = [float(x) for x in theta]
    assert len(theta) == 4
    hy = 1.5 * dx if half[1] is None else half[1]
    return dict(kind="plate", theta=theta, centre=[float(x) for x in centre],
                half=[float(half[0]), float(hy), float(half[2])],
                period=float(period))


def spheres_scene(seed, count=64, rmin=0.02, rmax=0.08):
    """``count`` static spheres, centres U[0,1]^3 and radii U[rmin, rmax]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.uniform(0.0, 1.0, size=(count, 3))
    r = rng.uniform(rmin, rmax, size=(count,))
    return dict(kind="spheres", theta=[],
                spheres=[[float(a), float(b), float(e), float(f)]
                         for (a, b, e), f in zip(c, r)])


def empty_scene():
    return dict(kind="none", theta=[])


def extruded_scene(seed, *, shapes=1, segments=5, keys=2, fluid="outside",
                   centre=(0.5, 0.5), radius=(0.14, 0.22), z=(0.3, 0.7)):
    """Static polar-Bezier shapes extruded along z (seeded radii).

    Each shape has ``keys`` key cross-sections of ``segments`` cubic
    segments; ``theta`` lists every radius, shape by shape, key by key, as
    rho1_0, rho2_0, rho1_1, ... . ``fluid`` says whether the fluid is outside
    the shapes (obstacles) or inside them (containers).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out, theta = [], []
    for k in range(shapes):
        cx = centre[0] + 0.12 * (k - (shapes - 1) / 2)
        ks = []
        for _ in range(keys):
            r = rng.uniform(radius[0], radius[1], size=2 * segments)
            theta += [float(v) for v in r]
            ks.append(dict(c=[float(cx), float(centre[1])], nseg=int(segments)))
        out.append(dict(z0=float(z[0]), z1=float(z[1]), keys=ks))
    return dict(kind="extruded", theta=theta, shapes=out, fluid=str(fluid))


def _frame(origin, z_dir):
    """A rigid frame whose local z is the unit vector along ``z_dir``."""
    z = np.asarray(z_dir, dtype=np.float64)
    z = z / np.linalg.norm(z)
    a = np.array([1.0, 0.0, 0.0]) if abs(z[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    x = np.cross(a, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return dict(origin=[float(v) for v in origin], axes=[list(map(float, r)) for r in (x, y, z)])


def heart_scene(seed, *, segments=5, pulse_period=None, outlet=False):
    """A heart-like container: the union of a chamber and three tubes (two
    inlets from the top, one outlet), each an extruded polar-Bezier shape in
    its own frame, the fluid inside the union.

    Static (default): theta lists every radius (chamber keys, then each
    tube's keys). With ``pulse_period`` the chamber contracts: its radii are
    k(t) times seeded base radii, k piecewise linear through 4 knots at t =
    0, T/3, 2T/3, T, and theta is those 4 knots (seeded near 1). With
    ``outlet`` the outlet tube runs along +x through the high-x wall (pair it
    with an outlet patch there); otherwise it ends inside the box.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes, radii = [], []

    def add(frame, z0, z1, centre, radius, keys):
        ks = []
        for _ in range(keys):
            r = rng.uniform(radius[0], radius[1], size=2 * segments)
            radii.extend(float(v) for v in r)
            ks.append(dict(c=[float(centre[0]), float(centre[1])], nseg=int(segments),
                           rho=[float(v) for v in r]))
        sh = dict(z0=float(z0), z1=float(z1), keys=ks)
        if frame is not None:
            sh["frame"] = frame
        shapes.append(sh)

    add(None, 0.3, 0.7, (0.5, 0.5), (0.16, 0.22), 3)                   # chamber
    add(_frame((0.42, 0.5, 0.5), (-0.3, 0.0, 1.0)), 0.0, 0.45, (0.0, 0.0), (0.05, 0.06), 2)
    add(_frame((0.58, 0.5, 0.5), (0.3, 0.0, 1.0)), 0.0, 0.45, (0.0, 0.0), (0.05, 0.06), 2)
    if outlet:
        add(_frame((0.5, 0.5, 0.5), (1.0, 0.0, 0.0)), 0.0, 0.65, (0.0, 0.0), (0.10, 0.11), 2)
    else:
        add(_frame((0.5, 0.5, 0.45), (0.0, 1.0, 0.0)), 0.0, 0.45, (0.0, 0.0), (0.06, 0.07), 2)
    sc = dict(kind="extruded", shapes=shapes, fluid="inside")
    if pulse_period is None:
        sc["theta"] = radii
    else:
        sc["theta"] = [float(v) for v in rng.uniform(0.85, 1.0, size=4)]
        sc["params"] = "pulse"
        sc["pulse"] = dict(shape=0, period=float(pulse_period))
    return sc


def shell_scene(lo, hi, thickness, v):
    """Hollow axis-aligned box shell translating with velocity ``v``.

    Solid between the boxes ``[lo, hi]`` and ``[lo + thickness, hi -
    thickness]``; used by the invariant test of the step (interior fluid
    moving with the shell stays uniform).
    """
    return dict(kind="shell", theta=[float(x) for x in v],
                lo=[float(x) for x in lo], hi=[float(x) for x in hi],
                thickness=float(thickness))


# --------------------------------------------------------------- configs ----

def config_sphere(n=32, *, seed=0, steps=20, dt=0.01, sigma=0.1, tol=1e-10):
    """Plain FP64 method: translating sphere in a closed box (32^3, 20 steps)."""
    g = make_grid(n, dt)
    return dict(name=f"sphere{n}", grid=g, scene=sphere_scene(),
                u0=gaussian_faces(g, sigma, seed), project_initial=True,
                steps=steps, tol=tol, loss="kinetic_energy")


def config_chamber(n=128, *, seed=0, steps=100, dt=0.005, tol=1e-6,
                   duct_half_cells=8, cfl_max=8.0):
    """Pulsing chamber with one outlet patch (128^3, 100 frames of dt).

    Each frame is split into steps under the CFL rule with ``cfl_max``
    (0 disables sub-stepping: one step per frame).
    """
    g = make_grid(n, dt, outlet=centred_outlet(n, 2 * duct_half_cells))
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.uniform(-0.05, 0.05, size=8)
    sc = chamber_scene(theta, g["dx"], duct_half_cells=duct_half_cells)
    return dict(name=f"chamber{n}", grid=g, scene=sc, u0=zero_faces(g),
                project_initial=False, steps=steps, tol=tol, loss="outflow",
                cfl_max=float(cfl_max))


def config_plate(n=64, *, seed=0, steps=16, dt=0.01, sigma=0.1, tol=1e-10):
    """Rotating plate with 4 angle knots (64^3, 16 steps)."""
    g = make_grid(n, dt)
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.uniform(-0.5, 0.5, size=4)
    sc = plate_scene(theta, g["dx"], period=steps * dt)
    return dict(name=f"plate{n}", grid=g, scene=sc,
                u0=gaussian_faces(g, sigma, seed + 1000), project_initial=True,
                steps=steps, tol=tol, loss="kinetic_energy")


def config_spheres(n=256, *, seed=0, count=64, tol=1e-8):
    """Single projection: 64 static spheres, divergent N(0, 1) velocity."""
    g = make_grid(n, 0.01)
    return dict(name=f"spheres{n}", grid=g, scene=spheres_scene(seed, count),
                u0=gaussian_faces(g, 1.0, seed + 2000), project_initial=True,
                steps=0, tol=tol, loss="kinetic_energy")


def serving_mix(seed=0, count=512, rate_per_ms=0.5,
                sizes=(32, 64, 96, 128, 192), adjoint_frac=0.3):
    """Seeded serving workload: Poisson arrivals of episode requests.

    Returns a list of dicts ``{arrival_ms, n, scene_kind, adjoint, seed}``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_ms, size=count)
    t = np.cumsum(gaps)
    out = []
    kinds = ("sphere", "chamber", "plate")
    for i in range(count):
        out.append(dict(arrival_ms=float(t[i]),
                        n=int(sizes[rng.integers(len(sizes))]),
                        scene_kind=kinds[rng.integers(3)],
                        adjoint=bool(rng.uniform() < adjoint_frac),
                        seed=int(rng.integers(1 << 31))))
    return out
