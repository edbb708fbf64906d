"""Pins of the oracle's geometry and rasteriser (no GPU)."""

import numpy as np
import pytest

import nf_inputs as I
from oracle import Grid, geometry, mac, rasterize


def _halfspace(axis, x0):
    """A plate scene whose only face inside the unit box is the plane
    ``x_axis = x0`` (solid below it): phi = x_axis - x0 there exactly."""
    centre = [0.5, 0.5, 0.5]
    centre[axis] = x0 - 10.0
    sc = I.plate_scene([0.0, 0.0, 0.0, 0.0], 0.1, 1.0, centre=centre, half=(10.0, 10.0, 10.0))
    sc["half"] = [10.0, 10.0, 10.0]
    return sc


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("x0", [0.3037, 0.5, 0.71])
def test_plane_fraction_is_exact_volume_fraction(axis, x0):
    # For an axis-aligned plane the 4-sample ramp average equals the exact
    # fluid fraction of the face's dx^3 control volume.
    g = Grid(I.make_grid(10, 0.01))
    alpha = rasterize.fractions(g, _halfspace(axis, x0), 0.0)
    for d in range(3):
        xf = mac.face_positions(g, d)[..., axis] * g.dx
        exact = np.clip((xf + 0.5 * g.dx - x0) / g.dx, 0.0, 1.0)
        interior = ~mac.boundary_face_mask(g, d)
        np.testing.assert_allclose(alpha[d][interior], exact[interior], atol=1e-12)
        assert np.all(alpha[d][~interior] == 0.0)


def test_fractions_saturate_away_from_the_interface():
    g = Grid(I.make_grid(16, 0.01))
    sc = I.sphere_scene()
    alpha = rasterize.fractions(g, sc, 0.0)
    for d in range(3):
        x = mac.face_positions(g, d) * g.dx
        ph = geometry.phi(sc, x, 0.0)
        interior = ~mac.boundary_face_mask(g, d)
        far_fluid = interior & (ph > 0.9 * g.dx)
        deep = interior & (ph < -0.9 * g.dx)
        assert far_fluid.any() and deep.any()
        assert np.all(alpha[d][far_fluid] == 1.0)
        assert np.all(alpha[d][deep] == 0.0)


def test_fluid_volume_converges_to_analytic():
    errs = []
    for n in (8, 16, 32):
        g = Grid(I.make_grid(n, 0.01))
        alpha = rasterize.fractions(g, I.sphere_scene(radius=0.2), 0.0)
        vol = alpha[0][:, :, 1:-1].sum() * g.dx ** 3
        exact = (1.0 - g.dx) - 4.0 / 3.0 * np.pi * 0.2 ** 3
        errs.append(abs(vol - exact))
    assert errs[-1] < 2e-4
    assert errs[2] < errs[0]


def test_outlet_and_wall_overrides():
    cfg = I.config_chamber(16, duct_half_cells=2)
    g = Grid(cfg["grid"])
    alpha = rasterize.fractions(g, cfg["scene"], 0.0)
    us = rasterize.face_solid_velocity(g, cfg["scene"], 0.01)
    out = mac.outlet_face_mask(g, 0)
    assert out.sum() == 16
    assert np.all(alpha[0][out] == 1.0)
    for d in range(3):
        wall = mac.boundary_face_mask(g, d) & ~mac.outlet_face_mask(g, d)
        assert np.all(alpha[d][wall] == 0.0)
        assert np.all(us[d][mac.boundary_face_mask(g, d)] == 0.0)


@pytest.mark.parametrize("cfgname", ["sphere", "chamber", "plate"])
def test_fraction_parameter_gradient_matches_finite_differences(cfgname):
    cfg = {"sphere": lambda: I.config_sphere(10),
           "chamber": lambda: I.config_chamber(12, duct_half_cells=2),
           "plate": lambda: I.config_plate(12)}[cfgname]()
    g = Grid(cfg["grid"])
    sc = cfg["scene"]
    t = 0.7 * (sc.get("period", 0.1))
    _, dalpha = rasterize.fractions(g, sc, t, with_grad=True)
    us, dus = rasterize.face_solid_velocity(g, sc, t, with_grad=True)
    th = np.array(sc["theta"])
    h = 1e-6
    rng = np.random.default_rng(0)
    w = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    for k in range(len(th)):
        sp, sm = dict(sc), dict(sc)
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        sp["theta"], sm["theta"] = list(tp), list(tm)
        ap, am = rasterize.fractions(g, sp, t), rasterize.fractions(g, sm, t)
        up, um = rasterize.face_solid_velocity(g, sp, t), rasterize.face_solid_velocity(g, sm, t)
        fd_a = sum(np.sum(w[d] * (ap[d] - am[d])) for d in range(3)) / (2 * h)
        an_a = sum(np.sum(w[d] * dalpha[d][..., k]) for d in range(3))
        fd_u = sum(np.sum(w[d] * (up[d] - um[d])) for d in range(3)) / (2 * h)
        an_u = sum(np.sum(w[d] * dus[d][..., k]) for d in range(3))
        assert abs(fd_a - an_a) <= 1e-5 * max(1.0, abs(an_a))
        assert abs(fd_u - an_u) <= 1e-6 * max(1.0, abs(an_u))


def test_solid_velocity_of_rigid_scenes_is_discretely_divergence_free():
    # rigid motions have zero discrete divergence cell by cell, which is what
    # makes the closed-box systems consistent
    for sc, t in ((I.sphere_scene(), 0.1), (I.plate_scene([0.1, -0.3, 0.4, 0.2], 1 / 12, 0.16), 0.07)):
        g = Grid(I.make_grid(12, 0.01))
        us = [geometry.solid_velocity(sc, mac.face_positions(g, d) * g.dx, t)[..., d] for d in range(3)]
        div = mac.grad_T(g, us)
        # boundary faces are not zeroed here: pure rigid field
        assert np.max(np.abs(div)) < 1e-13


# ---------------------------------------- corner (face-area) fractions ----
# The paper's own rule (Sec. 2.3.1, Projection): alpha is the fluid share of
# the face area bounded by the zero contour, whose crossings with the face
# edges come from phi at the corners.

def _corner(ph):
    return rasterize.corner_fraction(np.asarray(ph, dtype=np.float64))


@pytest.mark.parametrize("rot", [0, 1, 2, 3])
def test_corner_rule_reproduces_the_papers_single_corner_formula(rot):
    # one fluid corner A with neighbours B and D along the two face edges:
    # alpha = 1/2 phi_A / (phi_A - phi_B) * phi_A / (phi_A - phi_D)
    rng = np.random.default_rng(rot)
    for _ in range(50):
        pa = rng.uniform(0.01, 1.0)
        others = -rng.uniform(0.01, 1.0, size=3)
        ph = np.roll(np.concatenate([[pa], others]), rot)
        a = rot % 4
        pb, pd = ph[(a + 1) % 4], ph[(a + 3) % 4]
        want = 0.5 * pa / (pa - pb) * pa / (pa - pd)
        assert abs(_corner(ph)[0] - want) <= 1e-15


def test_corner_rule_is_exact_for_a_linear_phi():
    # a planar interface crosses the face in a straight line, so the linear
    # edge crossings are exact: alpha = the area where phi > 0, measured by
    # a dense midpoint count
    rng = np.random.default_rng(4)
    m = 2000
    s = (np.arange(m) + 0.5) / m
    S, T = np.meshgrid(s, s, indexing="ij")
    for _ in range(12):
        a0, b, c = rng.uniform(-1.0, 1.0, size=3)
        ph = [a0, a0 + b, a0 + b + c, a0 + c]       # corners (0,0) (1,0) (1,1) (0,1)
        want = np.mean(a0 + b * S + c * T > 0.0)
        assert abs(_corner(ph)[0] - want) <= 2e-3


def test_corner_rule_complement_and_saturation():
    rng = np.random.default_rng(5)
    assert _corner([1, 2, 3, 4])[0] == 1.0
    assert _corner([-1, -2, -3, -4])[0] == 0.0
    n = 0
    while n < 200:
        ph = rng.uniform(-1.0, 1.0, size=4)
        saddle = (ph[0] > 0) == (ph[2] > 0) and (ph[1] > 0) == (ph[3] > 0) and (ph[0] > 0) != (ph[1] > 0)
        if saddle:
            # two diagonal fluid corners: the fluid is connected, the two
            # solid corners are cut off as triangles
            sol = [c for c in range(4) if ph[c] < 0]
            tri = sum(0.5 * ph[c] / (ph[c] - ph[(c + 1) % 4]) * ph[c] / (ph[c] - ph[(c + 3) % 4])
                      for c in sol)
            assert abs(_corner(ph)[0] - (1.0 - tri)) <= 1e-14
            continue
        # no saddle: the solid part of phi is the fluid part of -phi
        assert abs(_corner(ph)[0] + _corner(-ph)[0] - 1.0) <= 1e-14
        n += 1


def test_corner_rule_gradient_matches_finite_differences():
    rng = np.random.default_rng(6)
    h = 1e-7
    for _ in range(100):
        ph = rng.uniform(-1.0, 1.0, size=4)
        ph[np.abs(ph) < 0.05] = 0.3                  # keep the sign pattern under the step
        _, g = _corner(ph)
        for c in range(4):
            e = np.zeros(4)
            e[c] = h
            fd = (_corner(ph + e)[0] - _corner(ph - e)[0]) / (2 * h)
            assert abs(fd - g[c]) <= 1e-6 * max(1.0, abs(g[c]))


def test_corner_rule_cross_section_of_a_sphere_converges():
    # the x faces of the plane through the sphere's centre carry the fluid
    # area 1 - pi r^2 of that plane (in units of the box face)
    errs = []
    for n in (16, 32, 64):
        g = Grid(dict(I.make_grid(n, 0.01), fractions="corner"))
        alpha = rasterize.fractions(g, I.sphere_scene(radius=0.2), 0.0)
        area = alpha[0][:, :, n // 2].sum() * g.dx ** 2
        errs.append(abs(area - (1.0 - np.pi * 0.2 ** 2)))
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs
    assert errs[2] < 3e-4


@pytest.mark.parametrize("cfgname", ["sphere", "plate"])
def test_corner_rule_parameter_gradient_matches_finite_differences(cfgname):
    cfg = {"sphere": lambda: I.config_sphere(10),
           "plate": lambda: I.config_plate(12)}[cfgname]()
    g = Grid(dict(cfg["grid"], fractions="corner"))
    sc = cfg["scene"]
    t = 0.7 * (sc.get("period", 0.1))
    _, dalpha = rasterize.fractions(g, sc, t, with_grad=True)
    th = np.array(sc["theta"])
    h = 1e-6
    rng = np.random.default_rng(1)
    w = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    seen = 0.0
    for k in range(len(th)):
        sp, sm = dict(sc), dict(sc)
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        sp["theta"], sm["theta"] = list(tp), list(tm)
        ap, am = rasterize.fractions(g, sp, t), rasterize.fractions(g, sm, t)
        fd = sum(np.sum(w[d] * (ap[d] - am[d])) for d in range(3)) / (2 * h)
        an = sum(np.sum(w[d] * dalpha[d][..., k]) for d in range(3))
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an))
        seen = max(seen, abs(an))
    assert seen > 1e-3          # the parameters do move the interface
