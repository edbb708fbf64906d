"""Pins of the oracle's MAC-grid operators (no GPU)."""

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import nf_inputs as I
from oracle import Grid
from oracle import mac


def _grid(n=6, ny=5, nz=4, periodic=False):
    return Grid(I.make_grid(n, 0.01, ny=ny, nz=nz, periodic=periodic))


def test_divergence_of_linear_field_is_closed_form():
    # G^T U = -dx * div(u); for u = (a x, b y, c z) on a closed box the
    # discrete divergence is exactly a + b + c in every cell.
    g = _grid()
    a, b, c = 0.7, -1.3, 2.1
    X = [mac.face_positions(g, d) * g.dx for d in range(3)]
    U = [a * X[0][..., 0], b * X[1][..., 1], c * X[2][..., 2]]
    div = -mac.grad_T(g, U) / g.dx
    np.testing.assert_allclose(div, a + b + c, rtol=0, atol=1e-12)


@pytest.mark.parametrize("periodic", [False, True])
def test_gradient_of_linear_pressure(periodic):
    g = _grid(periodic=periodic)
    Xc = np.stack(np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx),
                              indexing="ij"), -1)[..., ::-1] + 0.5
    P = 0.3 * Xc[..., 0] - 0.2 * Xc[..., 1] + 0.9 * Xc[..., 2]
    GP = mac.grad(g, P)
    # interior faces see the constant increments 0.3, -0.2, 0.9
    np.testing.assert_allclose(GP[0][:, :, 1:-1] if not periodic else GP[0][:, :, 1:], 0.3, atol=1e-12)
    np.testing.assert_allclose(GP[1][:, 1:-1, :] if not periodic else GP[1][:, 1:, :], -0.2, atol=1e-12)
    np.testing.assert_allclose(GP[2][1:-1] if not periodic else GP[2][1:], 0.9, atol=1e-12)
    if not periodic:
        # ghost pressure is zero outside the box
        np.testing.assert_allclose(GP[0][:, :, 0], P[:, :, 0])
        np.testing.assert_allclose(GP[0][:, :, -1], -P[:, :, -1])


@pytest.mark.parametrize("periodic", [False, True])
def test_trilinear_matches_library_interpolator(periodic):
    g = _grid(7, 6, 5, periodic=periodic)
    rng = np.random.default_rng(3)
    U = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    for e in range(3):
        npts = mac.lattice_points(g, e)
        shift = np.full(3, 0.5)
        shift[e] = 0.0
        axes = [np.arange(npts[a]) + shift[a] for a in range(3)]
        vals = U[e]
        if periodic:    # extend by one period for the library routine
            axes = [np.arange(npts[a] + 1) + shift[a] for a in range(3)]
            vals = np.pad(vals, [(0, 1)] * 3, mode="wrap")
        f = RegularGridInterpolator((axes[2], axes[1], axes[0]), vals)
        lo = np.array([ax[0] for ax in axes])
        hi = np.array([ax[-1] for ax in axes])
        X = lo + rng.uniform(0, 1, size=(200, 3)) * (hi - lo)
        ref = f(X[:, ::-1])
        np.testing.assert_allclose(mac.trilinear(g, e, U[e], X), ref, rtol=1e-12, atol=1e-12)


def test_trilinear_clamps_to_lattice_box():
    g = _grid()
    rng = np.random.default_rng(4)
    U = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    X = rng.uniform(-3, 10, size=(300, 3))
    for e in range(3):
        npts = mac.lattice_points(g, e)
        shift = np.full(3, 0.5)
        shift[e] = 0.0
        Xc = np.clip(X - shift, 0, np.array(npts) - 1) + shift
        np.testing.assert_allclose(mac.trilinear(g, e, U[e], X), mac.trilinear(g, e, U[e], Xc), atol=1e-14)


def test_trilinear_gradient_matches_finite_differences():
    g = _grid()
    rng = np.random.default_rng(5)
    U = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    X = rng.uniform(1.0, 3.9, size=(100, 3))
    h = 1e-7
    for e in range(3):
        gr = mac.trilinear_grad(g, e, U[e], X)
        for a in range(3):
            dX = np.zeros(3)
            dX[a] = h
            fd = (mac.trilinear(g, e, U[e], X + dX) - mac.trilinear(g, e, U[e], X - dX)) / (2 * h)
            np.testing.assert_allclose(gr[:, a], fd, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("periodic", [False, True])
def test_scatter_is_transpose_of_gather(periodic):
    g = _grid(periodic=periodic)
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 8, size=(50, 3))
    for e in range(3):
        u = rng.standard_normal(g.face_shape(e))
        w = rng.standard_normal(50)
        t = np.zeros_like(u)
        mac.trilinear_scatter(g, e, t, X, w)
        assert abs(np.dot(mac.trilinear(g, e, u, X), w) - np.sum(t * u)) < 1e-12
