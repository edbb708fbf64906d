"""Pins of the oracle's semi-Lagrangian advection and its adjoint (no GPU)."""

import numpy as np
import pytest

import nf_inputs as I
from oracle import Grid, advect, mac


def test_uniform_field_is_reproduced_with_clamping():
    g = Grid(I.make_grid(8, 0.05, ny=6, nz=5))
    V = (0.7, -0.4, 0.25)
    U = [np.full(g.face_shape(d), V[d]) for d in range(3)]
    Ut = advect.advect(g, U)
    for d in range(3):
        np.testing.assert_allclose(Ut[d], V[d], rtol=0, atol=1e-15)


@pytest.mark.parametrize("m", [1, 2, -3])
def test_periodic_shear_flow_shifts_exactly(m):
    # u = (V, f(x), 0) with V dt = m dx: the y component is carried exactly
    # m cells downstream, the x component stays V.
    n = 12
    g = Grid(I.make_grid(n, 0.01, ny=6, nz=4, periodic=True))
    V = m * g.dx / g.dt
    rng = np.random.default_rng(1)
    f = rng.standard_normal(n)
    U = g.zeros_faces()
    U[0][...] = V
    U[1][...] = f[None, None, :]
    Ut = advect.advect(g, U)
    np.testing.assert_allclose(Ut[0], V, atol=1e-12)
    np.testing.assert_allclose(Ut[1], np.roll(f, m)[None, None, :] * np.ones_like(U[1]), atol=1e-12)
    np.testing.assert_allclose(Ut[2], 0.0, atol=1e-15)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("periodic", [False, True])
def test_adjoint_matches_directional_derivative(order, periodic):
    g = Grid(I.make_grid(6, 0.02, ny=5, nz=4, periodic=periodic))
    rng = np.random.default_rng(2)
    U = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    dU = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    W = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    h = 1e-6
    up = advect.advect(g, [u + h * v for u, v in zip(U, dU)], order)
    um = advect.advect(g, [u - h * v for u, v in zip(U, dU)], order)
    jvp = sum(np.sum(w * (a - b)) for w, a, b in zip(W, up, um)) / (2 * h)
    gU = advect.advect_adjoint(g, U, W, order)
    vjp = sum(np.sum(a * b) for a, b in zip(gU, dU))
    assert abs(jvp - vjp) <= 1e-7 * abs(vjp)


def test_viscosity_adjoint_matches_directional_derivative():
    g = Grid(I.make_grid(6, 0.01, periodic=True, nu=0.3))
    rng = np.random.default_rng(3)
    U = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    W = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    lhs = sum(np.sum(w * v) for w, v in zip(W, advect.viscosity(g, U)))
    rhs = sum(np.sum(u * v) for u, v in zip(U, advect.viscosity_adjoint(g, W)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_viscosity_decays_a_fourier_mode_at_the_discrete_rate():
    # explicit Euler on sin(2 pi k x): factor 1 - 4 nu dt/dx^2 sin^2(pi k dx)
    n = 16
    g = Grid(I.make_grid(n, 0.01, ny=4, nz=4, periodic=True, nu=0.05))
    X = mac.face_positions(g, 1)[..., 0] * g.dx
    U = g.zeros_faces()
    U[1] = np.sin(2 * np.pi * 3 * X)
    Uh = advect.viscosity(g, U)
    fac = 1 - 4 * g.nu * g.dt / g.dx ** 2 * np.sin(np.pi * 3 * g.dx) ** 2
    np.testing.assert_allclose(Uh[1], fac * U[1], atol=1e-13)


# Closed boxes: the face lattice of each component ends at the walls, so
# -G^T G is the graph Laplacian of a path along every axis. Its eigenvectors
# are the DCT-II modes cos(pi m (i + 1/2) / n) with eigenvalue
# 2 - 2 cos(pi m / n) (n lattice points on that axis), a closed form that a
# wrong end treatment, a wrong lattice size or a sign error all break.
@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("modes", [(0, 0, 0), (1, 0, 2), (3, 2, 1), (0, 5, 0)])
def test_closed_box_viscosity_scales_lattice_cosine_modes(d, modes):
    g = Grid(I.make_grid(7, 0.004, ny=6, nz=9, nu=0.02))
    shp = g.face_shape(d)                               # (z, y, x) points
    npts = (shp[2], shp[1], shp[0])                     # (x, y, z)
    idx = np.meshgrid(np.arange(shp[0]), np.arange(shp[1]), np.arange(shp[2]),
                      indexing="ij")
    pos = (idx[2], idx[1], idx[0])                      # x, y, z indices
    mode = np.ones(shp)
    lam = 0.0
    for a in range(3):
        mode = mode * np.cos(np.pi * modes[a] * (pos[a] + 0.5) / npts[a])
        lam += 2.0 - 2.0 * np.cos(np.pi * modes[a] / npts[a])
    U = g.zeros_faces()
    U[d] = mode
    Uh = advect.viscosity(g, U)
    k = g.nu * g.dt / g.dx ** 2
    np.testing.assert_allclose(Uh[d], (1.0 - k * lam) * mode, rtol=0, atol=1e-13)
    for e in range(3):
        if e != d:
            assert not np.any(Uh[e])


def test_closed_box_viscosity_conserves_each_component_and_is_self_adjoint():
    g = Grid(I.make_grid(6, 0.003, ny=5, nz=4, nu=0.1))
    rng = np.random.default_rng(11)
    U = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    W = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    Uh = advect.viscosity(g, U)
    # no flux through the lattice ends: every component keeps its sum
    for d in range(3):
        assert abs(np.sum(Uh[d]) - np.sum(U[d])) <= 1e-12 * np.sum(np.abs(U[d]))
    lhs = sum(np.sum(w * v) for w, v in zip(W, Uh))
    rhs = sum(np.sum(u * v) for u, v in zip(U, advect.viscosity_adjoint(g, W)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_closed_box_viscosity_matches_the_assembled_lattice_matrix():
    # brute force on a tiny box: G assembled edge by edge from the lattice's
    # neighbour pairs, U^ = (I - k G^T G) U~ as a dense product
    g = Grid(I.make_grid(3, 0.01, ny=2, nz=4, nu=0.05))
    k = g.nu * g.dt / g.dx ** 2
    rng = np.random.default_rng(5)
    for d in range(3):
        shp = g.face_shape(d)
        n = int(np.prod(shp))
        rows = []
        for p in np.ndindex(*shp):
            for ax in range(3):
                q = list(p)
                q[ax] += 1
                if q[ax] < shp[ax]:
                    r = np.zeros(n)
                    r[np.ravel_multi_index(p, shp)] = -1.0
                    r[np.ravel_multi_index(tuple(q), shp)] = 1.0
                    rows.append(r)
        G = np.array(rows)
        u = rng.standard_normal(shp)
        U = g.zeros_faces()
        U[d] = u
        want = (np.eye(n) - k * G.T @ G) @ u.ravel()
        np.testing.assert_allclose(advect.viscosity(g, U)[d].ravel(), want,
                                   rtol=0, atol=1e-14)
