"""Pins of the oracle's polar-Bezier shapes, extrusion and CSG (no GPU).

Appendix A: N cubic segments around a centre, inner control points at
2 pi / (3N) from the ends of each segment's angular range, endpoints at the
midpoint of the two control points around them; key cross-sections along z
interpolated by the polynomial through the keys; CSG union/intersection.
"""

import numpy as np
import pytest

from oracle import bezier as B

C0 = (0.5, 0.45)


def _random_shape(seed, N=5):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.18, 0.34, N), rng.uniform(0.18, 0.34, N)


@pytest.mark.parametrize("N", [3, 4, 6, 9])
def test_equal_radii_endpoints_and_segment_midpoints_in_closed_form(N):
    # equal radii rho: every endpoint is the midpoint of two control points
    # at radius rho, 4 pi / (3N) apart, so at radius rho cos(2 pi / (3N));
    # the segment's midpoint B(1/2) = (e0 + 3 p0 + 3 p1 + e1) / 8 lies on the
    # bisector at radius (2 rho cos(2pi/3N) cos(pi/N) + 6 rho cos(pi/3N)) / 8
    rho = 0.27
    C = B.control_points(C0, [rho] * N, [rho] * N)
    c = np.asarray(C0)
    k = np.cos(2 * np.pi / (3 * N))
    for i in range(N):
        e = C[i, 0] - c
        assert abs(np.linalg.norm(e) - rho * k) <= 1e-15
        dang = (np.arctan2(e[1], e[0]) - 2 * np.pi * i / N + np.pi) % (2 * np.pi) - np.pi
        assert abs(dang) <= 1e-12
        m = B.bezier(C[i], 0.5) - c
        want = (2 * rho * k * np.cos(np.pi / N) + 6 * rho * np.cos(np.pi / (3 * N))) / 8
        assert abs(np.linalg.norm(m) - want) <= 1e-15
    # closed and G1: each endpoint is shared and lies on its control line
    for i in range(N):
        n = (i + 1) % N
        assert np.array_equal(C[i, 3], C[n, 0])
        a, b = C[i, 2] - C[i, 3], C[n, 1] - C[n, 0]
        assert abs(a[0] * b[1] - a[1] * b[0]) <= 1e-15


def test_distance_matches_dense_sampling_of_the_curve():
    r1, r2 = _random_shape(1)
    C = B.control_points(C0, r1, r2)
    s = np.linspace(0.0, 1.0, 200001)
    pts = np.concatenate([B.bezier(C[i], s) for i in range(len(C))])
    rng = np.random.default_rng(2)
    for x in rng.uniform(0.0, 1.0, size=(40, 2)):
        want = np.min(np.linalg.norm(pts - x, axis=-1))
        assert abs(abs(B.shape2d_sdf(C0, r1, r2, x)) - want) <= 1e-9


def _winding(poly, x):
    v = poly - x
    ang = np.arctan2(v[:, 1], v[:, 0])
    d = np.diff(np.concatenate([ang, ang[:1]]))
    d = (d + np.pi) % (2 * np.pi) - np.pi
    return int(round(d.sum() / (2 * np.pi)))


def test_sign_matches_the_winding_number_of_a_dense_polygon():
    r1, r2 = _random_shape(3)
    C = B.control_points(C0, r1, r2)
    s = np.linspace(0.0, 1.0, 400, endpoint=False)
    poly = np.concatenate([B.bezier(C[i], s) for i in range(len(C))])
    rng = np.random.default_rng(4)
    n_in = 0
    for x in rng.uniform(0.0, 1.0, size=(300, 2)):
        d = B.shape2d_sdf(C0, r1, r2, x)
        if abs(d) < 1e-3:
            continue
        inside = _winding(poly, x) != 0
        assert (d < 0) == inside
        n_in += inside
    assert n_in > 20


def _green_area(C):
    # area enclosed by the closed piecewise cubic: 1/2 sum of the integral of
    # x y' - y x' over each segment, exact by 4-point Gauss-Legendre (degree 5)
    g, w = np.polynomial.legendre.leggauss(4)
    s, w = 0.5 * (g + 1.0), 0.5 * w
    tot = 0.0
    for P in C:
        pts = B.bezier(P, s)
        e0, p0, p1, e1 = P
        d = (3 * (1 - s) ** 2)[:, None] * (p0 - e0) + (6 * (1 - s) * s)[:, None] * (p1 - p0) \
            + (3 * s ** 2)[:, None] * (e1 - p1)
        tot += 0.5 * np.sum(w * (pts[:, 0] * d[:, 1] - pts[:, 1] * d[:, 0]))
    return tot


def test_area_by_signs_converges_to_the_enclosed_area():
    r1, r2 = _random_shape(5)
    C = B.control_points(C0, r1, r2)
    exact = _green_area(C)
    m = 100
    g = (np.arange(m) + 0.5) / m
    P = np.array([(x, y) for x in g for y in g])
    inside = np.sum(B.shape2d_sdf_many(C0, r1, r2, P) < 0)
    assert abs(inside / m ** 2 - exact) <= 0.01 * exact


def test_radius_gradient_matches_finite_differences():
    r1, r2 = _random_shape(6)
    N = len(r1)
    rng = np.random.default_rng(7)
    h = 1e-6
    checked = 0
    for x in rng.uniform(0.05, 0.95, size=(30, 2)):
        C = B.control_points(C0, r1, r2)
        ds = sorted(B.closest_on_segment(C[i], x)[0] for i in range(N))
        if ds[1] - ds[0] < 1e-3:        # near the medial axis: not differentiable
            continue
        _, g = B.shape2d_sdf(C0, r1, r2, x, with_grad=True)
        for j in range(2 * N):
            a1, a2, b1, b2 = r1.copy(), r2.copy(), r1.copy(), r2.copy()
            (a1 if j % 2 == 0 else a2)[j // 2] += h
            (b1 if j % 2 == 0 else b2)[j // 2] -= h
            fd = (B.shape2d_sdf(C0, a1, a2, x) - B.shape2d_sdf(C0, b1, b2, x)) / (2 * h)
            assert abs(fd - g[j]) <= 1e-7
        checked += 1
    assert checked > 20


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_key_interpolation_passes_through_keys_and_reproduces_polynomials(n):
    for k in range(n):
        u = k / (n - 1) if n > 1 else 0.3
        np.testing.assert_allclose(B.lagrange_weights(n, u), np.eye(n)[k] if n > 1 else [1.0],
                                   atol=1e-12)
    # any polynomial of degree < n is reproduced at every u
    rng = np.random.default_rng(n)
    coef = rng.standard_normal(n)
    uk = np.arange(n) / max(n - 1, 1)
    vals = np.polyval(coef[::-1], uk)
    for u in rng.uniform(0.0, 1.0, size=5):
        assert abs(B.lagrange_weights(n, u) @ vals - np.polyval(coef[::-1], u)) <= 1e-11


def _prism(N=5, seed=8, keys=1):
    r1, r2 = _random_shape(seed, N)
    return dict(z0=0.3, z1=0.7, keys=[dict(c=C0, rho1=r1, rho2=r2)] * keys)


def test_extrusion_of_equal_keys_is_a_capped_prism():
    sh = _prism(keys=3)
    k = sh["keys"][0]
    # inside the slab, far from the caps: the cross-section's own distance
    for xy in [(0.5, 0.45), (0.9, 0.1), (0.62, 0.4)]:
        d2 = B.shape2d_sdf(k["c"], k["rho1"], k["rho2"], xy)
        assert abs(B.extrude_sdf(sh, (*xy, 0.5)) - (d2 if d2 > -0.2 else -0.2)) <= 1e-12 \
            or d2 < -0.2
    # straight above the deep interior: the distance to the top cap
    d2 = B.shape2d_sdf(k["c"], k["rho1"], k["rho2"], C0)
    assert d2 < -0.1
    for z in (0.75, 0.9):
        assert abs(B.extrude_sdf(sh, (*C0, z)) - (z - 0.7)) <= 1e-12
    # past a side wall and above the cap: the corner distance
    x = (0.98, 0.45, 0.8)
    d2 = B.shape2d_sdf(k["c"], k["rho1"], k["rho2"], x[:2])
    assert abs(B.extrude_sdf(sh, x) - np.hypot(d2, 0.1)) <= 1e-12


def test_extrusion_gradient_matches_finite_differences():
    rng = np.random.default_rng(9)
    keys = []
    for _ in range(3):
        keys.append(dict(c=C0 + rng.uniform(-0.03, 0.03, 2), rho1=rng.uniform(0.2, 0.3, 4),
                         rho2=rng.uniform(0.2, 0.3, 4)))
    sh = dict(z0=0.2, z1=0.8, keys=keys)
    h = 1e-6
    for x in [(0.6, 0.5, 0.35), (0.3, 0.4, 0.62), (0.55, 0.2, 0.5), (0.5, 0.5, 0.85)]:
        _, g = B.extrude_sdf(sh, x, with_grad=True)
        j = 0
        for k in range(3):
            for q in range(8):
                sp = [dict(kk, rho1=np.array(kk["rho1"]), rho2=np.array(kk["rho2"])) for kk in keys]
                sm = [dict(kk, rho1=np.array(kk["rho1"]), rho2=np.array(kk["rho2"])) for kk in keys]
                name = "rho1" if q % 2 == 0 else "rho2"
                sp[k][name][q // 2] += h
                sm[k][name][q // 2] -= h
                fd = (B.extrude_sdf(dict(sh, keys=sp), x) - B.extrude_sdf(dict(sh, keys=sm), x)) / (2 * h)
                assert abs(fd - g[j]) <= 1e-7, (x, k, q)
                j += 1


def test_union_and_intersection_areas():
    # two shapes: areas by sign counts obey inclusion-exclusion, and a union
    # of two disjoint shapes has the sum of their enclosed areas
    a1, a2 = _random_shape(10, 4)
    m = 120
    g = (np.arange(m) + 0.5) / m
    ca, cb, cf = (0.3, 0.5), (0.45, 0.5), (1.3, 0.5)
    P = np.array([(x, y) for x in g for y in g])
    sa = B.shape2d_sdf_many(ca, 0.6 * a1, 0.6 * a2, P)
    sb = B.shape2d_sdf_many(cb, 0.6 * a2, 0.6 * a1, P)
    u, i = B.union(sa, sb), B.intersection(sa, sb)
    assert (u < 0).sum() + (i < 0).sum() == (sa < 0).sum() + (sb < 0).sum()
    assert (i < 0).sum() > 0                              # they overlap
    # the same shape twice, 1 apart along x, sampled on [0, 2] x [0, 1]
    exact = _green_area(B.control_points(ca, 0.6 * a1, 0.6 * a2))
    g2 = (np.arange(2 * m) + 0.5) / m
    P2 = np.array([(x, y) for x in g2 for y in g])
    near = B.shape2d_sdf_many(ca, 0.6 * a1, 0.6 * a2, P2)
    far = B.shape2d_sdf_many(cf, 0.6 * a1, 0.6 * a2, P2)
    uf = B.union(near, far)
    assert abs((uf < 0).sum() / m ** 2 - 2 * exact) <= 0.03 * 2 * exact


def test_batched_evaluation_equals_the_point_by_point_one():
    r1, r2 = _random_shape(11, 6)
    rng = np.random.default_rng(12)
    X = rng.uniform(0.0, 1.0, size=(200, 2))
    sd, g = B.shape2d_sdf_many(C0, r1, r2, X, with_grad=True)
    for m in range(len(X)):
        d1, g1 = B.shape2d_sdf(C0, r1, r2, X[m], with_grad=True)
        assert abs(sd[m] - d1) <= 1e-12
        np.testing.assert_allclose(g[m], g1, atol=1e-10)
    keys = [dict(c=C0, rho1=r1, rho2=r2), dict(c=(0.52, 0.47), rho1=0.9 * r2, rho2=1.1 * r1)]
    sh = dict(z0=0.25, z1=0.75, keys=keys)
    X3 = np.concatenate([X[:40], rng.choice([0.1, 0.3, 0.5, 0.8], size=(40, 1))], axis=1)
    e, ge = B.extrude_sdf_many(sh, X3, with_grad=True)
    for m in range(len(X3)):
        e1, ge1 = B.extrude_sdf(sh, X3[m], with_grad=True)
        assert abs(e[m] - e1) <= 1e-12
        np.testing.assert_allclose(ge[m], ge1, atol=1e-10)


def test_sampled_newton_evaluation_equals_the_exact_one():
    # the rasteriser's evaluation (samples + Newton, normal side) against the
    # exact one (quintic roots, even-odd side), near and far from the curve
    rng = np.random.default_rng(13)
    keys = [dict(c=C0, rho1=rng.uniform(0.15, 0.3, 5), rho2=rng.uniform(0.15, 0.3, 5)),
            dict(c=(0.47, 0.5), rho1=rng.uniform(0.15, 0.3, 5), rho2=rng.uniform(0.15, 0.3, 5))]
    sh = dict(z0=0.2, z1=0.8, keys=keys)
    X = np.concatenate([rng.uniform(0.0, 1.0, size=(300, 2)), rng.uniform(0.1, 0.9, (300, 1))], 1)
    # points within 1e-3 of the curve: move random points onto it and off by a little
    k = keys[0]
    C = B.control_points(k["c"], k["rho1"], k["rho2"])
    near = np.array([B.bezier(C[rng.integers(5)], rng.uniform()) for _ in range(100)])
    near += rng.uniform(-1e-3, 1e-3, near.shape)
    X = np.concatenate([X, np.concatenate([near, np.full((100, 1), 0.2)], 1)])
    e, ge = B.extrude_sdf_many(sh, X, with_grad=True)
    for m in range(len(X)):
        e1, ge1 = B.extrude_sdf(sh, X[m], with_grad=True)
        assert abs(e[m] - e1) <= 1e-12, (m, X[m])
        np.testing.assert_allclose(ge[m], ge1, atol=1e-9)


# ------------------------------------------------ the extruded scene ----

def _prism_volume(sc):
    sh = sc["shapes"][0]
    th = np.asarray(sc["theta"])
    return _green_area(B.control_points(sh["keys"][0]["c"], th[0::2], th[1::2])) * (sh["z1"] - sh["z0"])


def test_extruded_obstacle_fluid_volume():
    import nf_inputs as I
    from oracle import Grid, rasterize
    sc = I.extruded_scene(3, shapes=1, keys=1)
    g = Grid(I.make_grid(8, 0.01))
    a = rasterize.fractions(g, sc, 0.0)
    # interior x-face control volumes cover [dx/2, 1 - dx/2] along x
    vol = a[0][:, :, 1:-1].sum() * g.dx ** 3
    V = _prism_volume(sc)
    assert abs(vol - ((1.0 - g.dx) - V)) <= 0.015 * V


@pytest.mark.parametrize("rule,n", [("corner", 10), ("supersample", 6)])
def test_extruded_scene_fraction_gradient_matches_finite_differences(rule, n):
    import nf_inputs as I
    from oracle import Grid, rasterize
    sc = I.extruded_scene(4, shapes=2, keys=2)
    g = Grid(dict(I.make_grid(n, 0.01), fractions=rule))
    _, dalpha = rasterize.fractions(g, sc, 0.0, with_grad=True)
    th = np.asarray(sc["theta"])
    rng = np.random.default_rng(14)
    w = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    h = 1e-6
    # a radius of each key of the two shapes (one for the slower rule)
    for k in ((0, 13, 27) if rule == "corner" else (27,)):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        ap = rasterize.fractions(g, dict(sc, theta=list(tp)), 0.0)
        am = rasterize.fractions(g, dict(sc, theta=list(tm)), 0.0)
        fd = sum(np.sum(w[d] * (ap[d] - am[d])) for d in range(3)) / (2 * h)
        an = sum(np.sum(w[d] * dalpha[d][..., k]) for d in range(3))
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (k, fd, an)
        assert abs(an) > 1e-3


# ------------------------------------------------ shapes in own frames ----

def _one_shape_scene(shape, r, fluid="outside"):
    return dict(kind="extruded", theta=list(r), shapes=[shape], fluid=fluid)


def test_a_framed_shape_is_the_unframed_one_in_local_coordinates():
    # frame rows: local x = world y, local y = world z, local z = world x
    # (a cyclic permutation, whose transpose is a different map)
    from oracle import geometry
    rng = np.random.default_rng(15)
    r = rng.uniform(0.1, 0.2, 10)
    base = dict(z0=0.2, z1=0.8, keys=[dict(c=[0.5, 0.45], nseg=5)])
    framed = dict(base, frame=dict(origin=[0.0, 0.0, 0.0],
                                   axes=[[0, 1, 0], [0, 0, 1], [1, 0, 0]]))
    X = rng.uniform(0.0, 1.0, size=(200, 3))
    a = geometry.phi(_one_shape_scene(framed, r), X, 0.0)
    b = geometry.phi(_one_shape_scene(base, r), X[:, [1, 2, 0]], 0.0)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_distance_is_constant_along_a_tilted_tube_axis():
    import nf_inputs as I
    from oracle import geometry
    rng = np.random.default_rng(16)
    r = rng.uniform(0.05, 0.07, 10)
    fr = I._frame((0.3, 0.4, 0.2), (1.0, 2.0, 2.0))
    tube = dict(z0=0.0, z1=0.6, keys=[dict(c=[0.0, 0.0], nseg=5)], frame=fr)
    d = np.asarray(fr["axes"][2])
    pts = np.asarray(fr["origin"]) + np.outer(np.linspace(0.15, 0.45, 7), d)
    ph = geometry.phi(_one_shape_scene(tube, r, fluid="inside"), pts, 0.0)
    assert np.all(ph > 0.03)
    assert np.ptp(ph) <= 1e-13


def test_heart_scene_fraction_gradient_matches_finite_differences():
    import nf_inputs as I
    from oracle import Grid, rasterize
    sc = I.heart_scene(2)
    g = Grid(dict(I.make_grid(12, 0.01), fractions="corner"))
    _, dalpha = rasterize.fractions(g, sc, 0.0, with_grad=True)
    th = np.asarray(sc["theta"])
    rng = np.random.default_rng(17)
    w = [rng.standard_normal(g.face_shape(d)) for d in range(3)]
    h = 1e-6
    for k in (3, 30, 75):            # a chamber radius, an inlet's, the outlet's
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        ap = rasterize.fractions(g, dict(sc, theta=list(tp)), 0.0)
        am = rasterize.fractions(g, dict(sc, theta=list(tm)), 0.0)
        fd = sum(np.sum(w[d] * (ap[d] - am[d])) for d in range(3)) / (2 * h)
        an = sum(np.sum(w[d] * dalpha[d][..., k]) for d in range(3))
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (k, fd, an)
        assert abs(an) > 1e-4, k


# ------------------------------------------------------ a pulsing heart ----

def _wall_points(sc, t, z=0.42):
    """Points on the pulsing chamber's side wall at time t (fluid side of
    the tubes' junctions: the -x half), where the chamber is the nearest."""
    from oracle import geometry
    sh = sc["shapes"][0]
    k = geometry.pulse_scale(sc, t)[0]
    n = len(sh["keys"])
    u = (z - sh["z0"]) / (sh["z1"] - sh["z0"])
    W = B.lagrange_weights(n, u)
    base = [np.asarray(kk["rho"]) for kk in sh["keys"]]
    r = k * sum(W[i] * base[i] for i in range(n))
    c = sum(W[i] * np.asarray(sh["keys"][i]["c"]) for i in range(n))
    C = B.control_points(c, r[0::2], r[1::2])
    pts = [np.append(B.bezier(C[i], s), z) for i in range(len(C)) for s in (0.3, 0.7)]
    return np.array([p for p in pts if p[0] < 0.45])


def test_pulsing_chamber_wall_moves_with_the_solid_velocity():
    # kinematic condition on the moving wall: d phi / dt + u_s . grad phi = 0
    import nf_inputs as I
    from oracle import geometry
    sc = I.heart_scene(5, pulse_period=0.06)
    t, h = 0.013, 1e-6
    X = _wall_points(sc, t)
    assert len(X) >= 3
    np.testing.assert_allclose(geometry.phi(sc, X, t), 0.0, atol=1e-12)
    dphidt = (geometry.phi(sc, X, t + h) - geometry.phi(sc, X, t - h)) / (2 * h)
    grad = np.stack([(geometry.phi(sc, X + h * e, t) - geometry.phi(sc, X - h * e, t)) / (2 * h)
                     for e in np.eye(3)], axis=-1)
    us = geometry.solid_velocity(sc, X, t)
    kdot = geometry.pulse_scale(sc, t)[1]
    assert abs(kdot) > 0.1
    np.testing.assert_allclose(dphidt + np.sum(us * grad, axis=-1), 0.0, atol=1e-6)


def test_pulsing_heart_phi_and_velocity_gradients_match_finite_differences():
    import nf_inputs as I
    from oracle import geometry
    sc = I.heart_scene(6, pulse_period=0.06, outlet=True)
    rng = np.random.default_rng(18)
    X = np.concatenate([_wall_points(sc, 0.031) + rng.uniform(-0.02, 0.02, (1, 3)),
                        rng.uniform(0.2, 0.8, size=(40, 3))])
    t, h = 0.031, 1e-6
    dphi = geometry.dphi_dtheta(sc, X, t)
    dus = geometry.dus_dtheta(sc, X, t)
    th = np.asarray(sc["theta"])
    for k in range(4):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        sp, sm = dict(sc, theta=list(tp)), dict(sc, theta=list(tm))
        fd = (geometry.phi(sp, X, t) - geometry.phi(sm, X, t)) / (2 * h)
        np.testing.assert_allclose(dphi[:, k], fd, atol=1e-7)
        fdu = (geometry.solid_velocity(sp, X, t) - geometry.solid_velocity(sm, X, t)) / (2 * h)
        np.testing.assert_allclose(dus[:, :, k], fdu, atol=1e-6)
    assert np.abs(dphi).max() > 1e-3 and np.abs(dus).max() > 1e-2
