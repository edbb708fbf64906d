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
