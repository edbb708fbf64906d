"""Pins of the oracle's full step, rollout and adjoint (no GPU)."""

import numpy as np
import pytest

import nf_inputs as I
from oracle import Grid, mac, project, rasterize
from oracle import step as S


# ------------------------------------------------------ Taylor-Green ----

def _taylor_green_ratio(n, nu=0.01, amp=1e-3, t_end=0.4):
    dt0 = 0.1 * (1.0 / n) ** 2 / nu
    steps = int(np.ceil(t_end / dt0))
    dt = t_end / steps
    g = Grid(I.make_grid(n, dt, nz=4, periodic=True, nu=nu))
    U = g.zeros_faces()
    X0 = mac.face_positions(g, 0) * g.dx
    X1 = mac.face_positions(g, 1) * g.dx
    tp = 2 * np.pi
    U[0] = amp * np.sin(tp * X0[..., 0]) * np.cos(tp * X0[..., 1])
    U[1] = -amp * np.cos(tp * X1[..., 0]) * np.sin(tp * X1[..., 1])
    U0 = [u.copy() for u in U]
    for k in range(steps):
        U, _ = S.step(g, I.empty_scene(), U, k, 1e-12)
    num = sum(np.sum(a * b) for a, b in zip(U, U0)) / sum(np.sum(b * b) for b in U0)
    return num, np.exp(-8 * np.pi ** 2 * nu * t_end)


def test_taylor_green_decay_converges_to_analytic():
    r16, ex = _taylor_green_ratio(16)
    r32, _ = _taylor_green_ratio(32)
    e16, e32 = abs(r16 - ex) / ex, abs(r32 - ex) / ex
    assert e32 < 0.02
    assert e32 < e16


# ----------------------------------------------------------- shell -----

def test_fluid_inside_a_translating_shell_moves_rigidly():
    n = 16
    g = Grid(I.make_grid(n, 0.02))
    V = np.array([0.3, -0.2, 0.1])
    sc = I.shell_scene((0.2, 0.2, 0.2), (0.8, 0.8, 0.8), 3.0 / n, V)
    U = g.zeros_faces()
    for d in range(3):
        X = mac.face_positions(g, d) * g.dx
        inside = np.all((X > 0.2) & (X < 0.8), axis=-1)
        U[d][inside] = V[d]
    for k in range(3):
        U, tape = S.step(g, sc, U, k, 1e-13)
    t = tape["t"]
    for d in range(3):
        X = mac.face_positions(g, d) * g.dx
        deep = np.all((X > 0.2 + V * t + 3.0 / n) & (X < 0.8 + V * t - 3.0 / n), axis=-1)
        assert deep.sum() > 20
        np.testing.assert_allclose(U[d][deep], V[d], rtol=0, atol=1e-12)


# --------------------------------------------------- projection adjoint ----

def _proj_case(seed=0):
    cfg = I.config_plate(10)
    g = Grid(cfg["grid"])
    alpha = rasterize.fractions(g, cfg["scene"], 0.05)
    us = rasterize.face_solid_velocity(g, cfg["scene"], 0.05)
    rng = np.random.default_rng(seed)
    Uh = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    W = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    return g, alpha, us, Uh, W, rng


def _dot(a, b):
    return sum(float(np.sum(x * y)) for x, y in zip(a, b))


def test_projection_adjoint_in_velocity_and_solid_velocity():
    g, alpha, us, Uh, W, rng = _proj_case(1)
    tol = 1e-14
    U0, P0, _ = project.project(g, alpha, us, Uh, tol)
    gUh, gS, gUs, y, _ = project.project_adjoint(g, alpha, us, Uh, P0, W, tol)
    dU = [rng.standard_normal(u.shape) for u in Uh]
    dUs = [rng.standard_normal(u.shape) * (~mac.boundary_face_mask(g, d)) for d, u in enumerate(us)]
    U1, _, _ = project.project(g, alpha, us, [a + b for a, b in zip(Uh, dU)], tol)
    lhs = _dot(W, [a - b for a, b in zip(U1, U0)])
    assert abs(lhs - _dot(gUh, dU)) <= 1e-9 * abs(lhs)
    U2, _, _ = project.project(g, alpha, [a + b for a, b in zip(us, dUs)], Uh, tol)
    lhs = _dot(W, [a - b for a, b in zip(U2, U0)])
    assert abs(lhs - _dot(gUs, dUs)) <= 1e-9 * abs(lhs)


def test_projection_adjoint_in_fractions():
    g, alpha, us, Uh, W, rng = _proj_case(2)
    tol = 1e-14
    U0, P0, _ = project.project(g, alpha, us, Uh, tol)
    _, gS, _, _, _ = project.project_adjoint(g, alpha, us, Uh, P0, W, tol)
    # perturb only cut faces, keeping the active set fixed
    dA = [rng.standard_normal(a.shape) * ((a > 0.05) & (a < 0.95)) for a in alpha]
    h = 1e-6
    Up, _, _ = project.project(g, [a + h * b for a, b in zip(alpha, dA)], us, Uh, tol)
    Um, _, _ = project.project(g, [a - h * b for a, b in zip(alpha, dA)], us, Uh, tol)
    fd = _dot(W, [a - b for a, b in zip(Up, Um)]) / (2 * h)
    assert abs(fd - _dot(gS, dA)) <= 1e-6 * abs(fd)


# ------------------------------------------------- rollout gradients ----

def _viscous(cfg, nu):
    cfg["grid"]["nu"] = float(nu)
    return cfg


def _corner(cfg):
    cfg["grid"]["fractions"] = "corner"
    return cfg


@pytest.mark.parametrize("name", ["sphere", "plate", "chamber", "sphere_viscous",
                                  "sphere_corner", "plate_corner"])
def test_rollout_gradient_matches_central_differences(name):
    # sphere_viscous: explicit viscosity with nu dt / dx^2 = 0.072 in the
    # closed box (Eq. viscosity_matrix and its adjoint, Sec. 2.3.2)
    cfg = {"sphere": lambda: I.config_sphere(12, steps=3),
           "plate": lambda: I.config_plate(12, steps=4),
           "chamber": lambda: I.config_chamber(16, steps=4, duct_half_cells=2),
           "sphere_viscous": lambda: _viscous(I.config_sphere(12, steps=3), 0.05),
           # the paper's face-area fractions from corner values (Sec. 2.3.1)
           "sphere_corner": lambda: _corner(I.config_sphere(12, steps=3)),
           "plate_corner": lambda: _corner(I.config_plate(12, steps=4))}[name]()
    J, g_adj, _ = S.loss_and_grad(cfg, tol=1e-12)
    g_fd = S.fd_gradient(cfg, h=1e-4, tol=1e-12)
    err = np.linalg.norm(g_adj - g_fd) / np.linalg.norm(g_fd)
    assert err < 1e-3, (g_adj, g_fd)


def test_extruded_obstacle_rollout_gradient_matches_central_differences():
    # polar-Bezier obstacles (App. A), corner fractions: the adjoint of a
    # two-step rollout against central differences in two of the radii
    g = I.make_grid(10, 0.01, nz=10)
    g["fractions"] = "corner"
    cfg = dict(name="extruded10", grid=g, scene=I.extruded_scene(4, shapes=2, keys=2),
               u0=I.gaussian_faces(g, 0.1, 21), project_initial=True, steps=2, tol=1e-12,
               loss="kinetic_energy")
    J, g_adj, _ = S.loss_and_grad(cfg, tol=1e-12)
    which = [0, 27]
    g_fd = S.fd_gradient(cfg, h=1e-5, tol=1e-12, which=which)
    for k in which:
        assert abs(g_adj[k] - g_fd[k]) <= 2e-3 * np.abs(g_fd[which]).max(), (k, g_adj[k], g_fd[k])
    assert np.abs(g_fd[which]).max() > 0.0


def _active_boundary_flux(g, alpha, us):
    """sum over faces with exactly one active neighbour (outlet excluded) of
    (a_high - a_low) u_s: by incompressibility this equals the outflow."""
    act = project.active_cells(g, alpha)
    tot = 0.0
    for d in range(3):
        ax = mac.axis_of(d)
        pad = [(0, 0)] * 3
        pad[ax] = (1, 1)
        a = np.pad(act, pad).astype(np.float64)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        sgn = a[tuple(hi)] - a[tuple(lo)]
        sgn[mac.outlet_face_mask(g, d)] = 0.0
        tot += float(np.sum(sgn * us[d]))
    return tot


def test_chamber_outflow_equals_geometric_volume_rate_and_its_gradient():
    cfg = I.config_chamber(16, steps=4, duct_half_cells=2)
    J, g_adj, info = S.loss_and_grad(cfg, tol=1e-13)
    g = Grid(cfg["grid"])
    t = cfg["steps"] * g.dt
    alpha = rasterize.fractions(g, cfg["scene"], t)
    us, dus = rasterize.face_solid_velocity(g, cfg["scene"], t, with_grad=True)
    geo = g.dx ** 2 * _active_boundary_flux(g, alpha, us)
    assert abs(J - geo) <= 1e-9 * abs(J)
    K = len(cfg["scene"]["theta"])
    g_geo = np.array([g.dx ** 2 * _active_boundary_flux(g, alpha, [dus[d][..., k] for d in range(3)])
                      for k in range(K)])
    np.testing.assert_allclose(g_adj, g_geo, rtol=1e-7, atol=1e-9 * np.abs(g_geo).max())


def test_pulsing_heart_outflow_equals_geometric_volume_rate_and_its_gradient():
    # the heart of Sec. 3 as a union of extruded polar-Bezier parts (App. A),
    # its chamber contracting by k(t) (4 control knots), one opening: the
    # outlet tube through the high-x patch. As for the chamber, the outflow
    # is the rate of change of the fluid volume, a function of alpha and u_s
    n = 12
    g0 = I.make_grid(n, 0.01, outlet=I.centred_outlet(n, 2))
    g0["fractions"] = "corner"
    cfg = dict(name="heart12", grid=g0, scene=I.heart_scene(7, pulse_period=0.06, outlet=True),
               u0=I.zero_faces(g0), project_initial=False, steps=2, tol=1e-13, loss="outflow")
    J, g_adj, _ = S.loss_and_grad(cfg, tol=1e-13)
    g = Grid(cfg["grid"])
    t = cfg["steps"] * g.dt
    alpha = rasterize.fractions(g, cfg["scene"], t)
    us, dus = rasterize.face_solid_velocity(g, cfg["scene"], t, with_grad=True)
    geo = g.dx ** 2 * _active_boundary_flux(g, alpha, us)
    assert abs(J) > 0.1
    assert abs(J - geo) <= 1e-9 * abs(J)
    g_geo = np.array([g.dx ** 2 * _active_boundary_flux(g, alpha, [dus[d][..., k] for d in range(3)])
                      for k in range(4)])
    np.testing.assert_allclose(g_adj, g_geo, rtol=1e-7, atol=1e-9 * np.abs(g_geo).max())


# ------------------------------------------------------- inflow patch ----

def test_uniform_through_flow_is_steady():
    # the whole low-x wall an inflow at speed V, the whole high-x wall open,
    # no solid: the uniform field V is divergence free and stays exactly
    n, V = 8, 0.37
    g0 = I.make_grid(n, 0.02, inlet=dict(axis=0, side=-1, j0=0, k0=0, w=n, h=n, speed=V),
                     outlet=dict(axis=0, side=1, j0=0, k0=0, w=n, h=n))
    g = Grid(g0)
    U = [np.full(g.face_shape(0), V), np.zeros(g.face_shape(1)), np.zeros(g.face_shape(2))]
    sc = dict(kind="none", theta=[])
    for k in range(3):
        U, _ = S.step(g, sc, U, k, 1e-13)
    # the y and z walls stay walls (u = 0); x faces carry V everywhere
    np.testing.assert_allclose(U[0], V, rtol=0, atol=1e-12)
    for d in (1, 2):
        np.testing.assert_allclose(U[d], 0.0, rtol=0, atol=1e-12)


def test_outflow_equals_inflow_past_a_moving_sphere():
    # incompressibility: the net flux out is the inflow, since a rigid
    # motion adds none; both patches 4 x 4 faces
    n, V = 16, 0.3
    cfg = I.config_sphere(n, steps=2)
    cfg["grid"] = I.make_grid(n, 0.01, inlet=I.centred_inlet(n, 4, V),
                              outlet=I.centred_outlet(n, 4))
    cfg["u0"] = I.gaussian_faces(cfg["grid"], 0.1, 3)
    cfg["loss"] = "outflow"
    g = Grid(cfg["grid"])
    U, _ = S.rollout(g, cfg["scene"], cfg["u0"], cfg["steps"], 1e-13, True)
    J, _ = S.outflow(g, U)
    assert abs(J - V * 16 * g.dx ** 2) <= 1e-10 * J


def test_rollout_gradient_with_an_inlet_matches_central_differences():
    n = 12
    cfg = I.config_sphere(n, steps=3)
    cfg["grid"] = I.make_grid(n, 0.01, inlet=I.centred_inlet(n, 4, 0.3),
                              outlet=I.centred_outlet(n, 4))
    cfg["u0"] = I.gaussian_faces(cfg["grid"], 0.1, 4)
    J, g_adj, _ = S.loss_and_grad(cfg, tol=1e-12)
    g_fd = S.fd_gradient(cfg, h=1e-4, tol=1e-12)
    err = np.linalg.norm(g_adj - g_fd) / np.linalg.norm(g_fd)
    assert err < 1e-3, (g_adj, g_fd)


# ------------------------------------------------- the 2D variant ----

def test_two_dimensional_channel_past_a_cylinder():
    # a 2D scene as a one-cell slab (nz = 1, closed z walls): uniform inflow
    # through the whole low-x wall, open high-x wall, a cylinder (an extruded
    # near-circular polar-Bezier shape through all z). u_z stays zero, the
    # outflow equals the inflow, and the flow keeps the mirror symmetry of
    # the cylinder and the data about the centre line y = 1/2
    n, V = 24, 0.3
    g0 = I.make_grid(n, 0.005, nz=1, inlet=dict(axis=0, side=-1, j0=0, k0=0, w=n, h=1, speed=V),
                     outlet=dict(axis=0, side=1, j0=0, k0=0, w=n, h=1))
    g0["fractions"] = "corner"
    sc = dict(kind="extruded", theta=[0.08] * 12, fluid="outside",
              shapes=[dict(z0=-1.0, z1=2.0, keys=[dict(c=[0.35, 0.5], nseg=6)])])
    g = Grid(g0)
    U0 = [np.full(g.face_shape(0), V), np.zeros(g.face_shape(1)), np.zeros(g.face_shape(2))]
    U, _ = S.rollout(g, sc, U0, 3, 1e-13, project_initial=True)
    assert not np.any(U[2])
    J, _ = S.outflow(g, U)
    assert abs(J - V * n * g.dx ** 2) <= 1e-12
    ux, uy = U[0][0], U[1][0]                  # (y, x) layers of the slab
    assert np.abs(uy).max() > 0.05             # the cylinder deflects the flow
    np.testing.assert_allclose(ux, ux[::-1, :], rtol=0, atol=1e-9)
    np.testing.assert_allclose(uy, -uy[::-1, :], rtol=0, atol=1e-9)


def test_substepped_chamber_keeps_the_outflow_identity():
    # CFL sub-stepping (Table 1: more steps than frames): the frame ends at
    # t = frames * dt whatever the split, so the final outflow still equals
    # the geometric volume rate at that time, and so does its gradient
    cfg = I.config_chamber(16, steps=3, duct_half_cells=2, cfl_max=1.0)
    J, g_adj, info = S.loss_and_grad(cfg, tol=1e-13)
    assert len(info["tapes"]) > cfg["steps"], "no frame was split"
    g = Grid(cfg["grid"])
    t = cfg["steps"] * g.dt
    assert abs(info["tapes"][-1]["t"] - t) <= 1e-15
    alpha = rasterize.fractions(g, cfg["scene"], t)
    us, dus = rasterize.face_solid_velocity(g, cfg["scene"], t, with_grad=True)
    geo = g.dx ** 2 * _active_boundary_flux(g, alpha, us)
    assert abs(J - geo) <= 1e-9 * abs(J)
    K = len(cfg["scene"]["theta"])
    g_geo = np.array([g.dx ** 2 * _active_boundary_flux(g, alpha, [dus[d][..., k] for d in range(3)])
                      for k in range(K)])
    np.testing.assert_allclose(g_adj, g_geo, rtol=1e-7, atol=1e-9 * np.abs(g_geo).max())
