"""Polar-Bezier shapes, their extrusion and CSG (oracle; tests only).

Appendix A (Geometry Representation) and Sec. 2.2. A closed 2D curve is N
cubic Bezier segments around a centre c. Segment i spans the polar angles
[2 pi i / N, 2 pi (i + 1) / N]. Its two inner control points sit at the
radii rho1_i and rho2_i, 2 pi / (3N) in from each end of that range. Its
endpoints are shared with the neighbouring segments, and each endpoint lies
on the line through the two control points around it (G1 continuity). That
fixes the line, not the point on it: the endpoint is read as the midpoint of
the two control points.

A 3D shape extrudes cross-sections along z between z0 and z1. The printed
interpolation of the key cross-sections is garbled (a power sum from i = 1
vanishes at z = z0). It is read as the polynomial in u = (z - z0) / (z1 -
z0), in power form, that passes through every key, with the n keys evenly
spaced, u_k = k / (n - 1). That interpolant is applied to the centre and to
each radius.

Signed distances here are positive outside the shape. The 2D distance is
the exact distance to the curve: the closest point of each segment is a root
of a quintic (NumPy's polynomial roots) or an end. The sign comes from the
even-odd count of the curve's crossings along a ray. The extrusion combines
the cross-section distance at the point's z with the slab |z - zm| <= h in
the usual capped form. CSG union and intersection are the min and max of the
distances (Sec. 2.2).

The scalar functions above are the definition. The many-point functions
give every point its own interpolated cross-section. They find the
closest parameter of each segment by Newton steps from the nearest of a few
samples, and take the side from the outward normal at the closest point.
This faster evaluation of the same distance serves the rasteriser, and the
tests hold it to the scalar one.
"""

from __future__ import annotations

import numpy as np


# ---------------------------------------------------------- 2D curve -----

def control_points(c, rho1, rho2):
    """Control polygons (N, 4, 2) of the closed curve: rows e0, p0, p1, e1."""
    c = np.asarray(c, dtype=np.float64)
    r1 = np.asarray(rho1, dtype=np.float64)
    r2 = np.asarray(rho2, dtype=np.float64)
    N = len(r1)
    base = 2.0 * np.pi * np.arange(N) / N
    a0 = base + 2.0 * np.pi / (3.0 * N)
    a1 = base + 4.0 * np.pi / (3.0 * N)
    p0 = c + r1[:, None] * np.stack([np.cos(a0), np.sin(a0)], axis=-1)
    p1 = c + r2[:, None] * np.stack([np.cos(a1), np.sin(a1)], axis=-1)
    e0 = 0.5 * (np.roll(p1, 1, axis=0) + p0)        # shared with segment i - 1
    e1 = np.roll(e0, -1, axis=0)
    return np.stack([e0, p0, p1, e1], axis=1)


def control_jacobian(N):
    """d(control polygon)/d(radius) as weights (N, 4, 2N): entry [i, r, j]
    is the factor by which row r of segment i moves along its radial unit
    vector when parameter j = (rho1_0, rho2_0, rho1_1, ...) changes.

    p0_i depends on rho1_i, p1_i on rho2_i, e0_i = (p1_{i-1} + p0_i) / 2."""
    J = np.zeros((N, 4, 2 * N))
    for i in range(N):
        J[i, 1, 2 * i] = 1.0
        J[i, 2, 2 * i + 1] = 1.0
        J[i, 0, 2 * ((i - 1) % N) + 1] = 0.5
        J[i, 0, 2 * i] = 0.5
        J[i, 3, 2 * i + 1] = 0.5
        J[i, 3, 2 * ((i + 1) % N)] = 0.5
    return J


def bernstein(s):
    s = np.asarray(s, dtype=np.float64)
    return np.stack([(1 - s) ** 3, 3 * (1 - s) ** 2 * s, 3 * (1 - s) * s ** 2, s ** 3], axis=-1)


def bezier(P, s):
    """Point(s) of the cubic with control polygon P (4, 2) at parameter s."""
    return bernstein(s) @ P


def _power(P):
    """Power-basis coefficients a0..a3 (4, 2) of the cubic: B = sum a_k s^k."""
    e0, p0, p1, e1 = P
    return np.array([e0, 3 * (p0 - e0), 3 * (e0 - 2 * p0 + p1), e1 - e0 + 3 * (p0 - p1)])


def closest_on_segment(P, x):
    """(distance, s*) from the 2D point x to the cubic P over s in [0, 1]."""
    a = _power(P)
    b = a.copy()
    b[0] = a[0] - x                                   # B(s) - x
    db = np.array([a[1], 2 * a[2], 3 * a[3]])          # B'(s)
    # (B - x) . B' as a degree-5 polynomial, coefficients in ascending order
    q = np.zeros(6)
    for i in range(4):
        for j in range(3):
            q[i + j] += b[i] @ db[j]
    cand = [0.0, 1.0]
    if np.any(q != 0.0):
        for r in np.roots(q[::-1]):
            if abs(r.imag) < 1e-9 and 0.0 < r.real < 1.0:
                cand.append(float(r.real))
    best = min(cand, key=lambda s: float(np.sum((bezier(P, s) - x) ** 2)))
    return float(np.linalg.norm(bezier(P, best) - x)), best


def _crossings(P, x):
    """Crossings of the ray from x towards +x with the cubic, s in [0, 1)."""
    a = _power(P)
    coef = [a[3][1], a[2][1], a[1][1], a[0][1] - x[1]]
    n = 0
    if not any(coef[:3]):
        return 0
    for r in np.roots(coef):
        if abs(r.imag) < 1e-12 and 0.0 <= r.real < 1.0:
            s = float(r.real)
            if bezier(P, s)[0] > x[0]:
                n += 1
    return n


def shape2d_sdf(c, rho1, rho2, x, with_grad=False):
    """Signed distance (positive outside) of the 2D point x to the closed
    curve, and optionally its gradient with respect to the 2N radii."""
    x = np.asarray(x, dtype=np.float64)
    C = control_points(c, rho1, rho2)
    N = len(C)
    best = (np.inf, 0, 0.0)
    for i in range(N):
        d, s = closest_on_segment(C[i], x)
        if d < best[0]:
            best = (d, i, s)
    d, i, s = best
    inside = sum(_crossings(C[k], x) for k in range(N)) % 2 == 1
    sd = -d if inside else d
    if not with_grad:
        return sd
    # envelope: d(dist)/d(rho_j) = -n . dB/d(rho_j) at the closest point,
    # n the unit vector from the curve to x
    foot = bezier(C[i], s)
    n = (x - foot) / d if d > 0.0 else np.zeros(2)
    # each control point moves along its own radial unit vector
    base = 2.0 * np.pi * np.arange(N) / N
    a0 = base + 2.0 * np.pi / (3.0 * N)
    a1 = base + 4.0 * np.pi / (3.0 * N)
    u0 = np.stack([np.cos(a0), np.sin(a0)], axis=-1)
    u1 = np.stack([np.cos(a1), np.sin(a1)], axis=-1)
    w = bernstein(s)
    grad = np.zeros(2 * N)
    J = control_jacobian(N)
    for r in range(4):
        for j in np.nonzero(J[i, r])[0]:
            k = j // 2
            u = u0[k] if j % 2 == 0 else u1[k]
            grad[j] += -(n @ u) * w[r] * J[i, r, j]
    return sd, (-grad if inside else grad)


# ------------------------------------------------------------ extrusion ----

def lagrange_weights(n, u):
    """Weights W (n,) with sum_k W_k v_k = the polynomial through the n keys
    (u_k = k / (n - 1)) at u, formed in power form: solve the Vandermonde
    system for the coefficients of each unit key vector."""
    if n == 1:
        return np.ones(1)
    uk = np.arange(n) / (n - 1)
    V = np.vander(uk, n, increasing=True)              # V[k, m] = u_k^m
    coeff = np.linalg.solve(V, np.eye(n))              # column k: key k alone
    powers = u ** np.arange(n)
    return powers @ coeff


def extrude_sdf(shape, x, with_grad=False):
    """Signed distance (positive outside) of the 3D point x to the extruded
    shape ``dict(z0, z1, keys=[dict(c=(cx, cy), rho1=[...], rho2=[...]), ...])``,
    optionally with the gradient with respect to every key's radii
    (ordered key by key, each as rho1_0, rho2_0, rho1_1, ...)."""
    x = np.asarray(x, dtype=np.float64)
    keys = shape["keys"]
    n = len(keys)
    z0, z1 = float(shape["z0"]), float(shape["z1"])
    u = np.clip((x[2] - z0) / (z1 - z0), 0.0, 1.0)
    W = lagrange_weights(n, u)
    c = sum(W[k] * np.asarray(keys[k]["c"], dtype=np.float64) for k in range(n))
    r1 = sum(W[k] * np.asarray(keys[k]["rho1"], dtype=np.float64) for k in range(n))
    r2 = sum(W[k] * np.asarray(keys[k]["rho2"], dtype=np.float64) for k in range(n))
    if with_grad:
        d, gd = shape2d_sdf(c, r1, r2, x[:2], with_grad=True)
    else:
        d = shape2d_sdf(c, r1, r2, x[:2])
    zm, h = 0.5 * (z0 + z1), 0.5 * (z1 - z0)
    w = abs(x[2] - zm) - h
    out = min(max(d, w), 0.0) + np.hypot(max(d, 0.0), max(w, 0.0))
    if not with_grad:
        return out
    # d(out)/d(d): 1 inside where d is the larger term; d+ / |(d+, w+)| outside
    if d <= 0.0 and w <= 0.0:
        dd = 1.0 if d >= w else 0.0
    else:
        dd = max(d, 0.0) / np.hypot(max(d, 0.0), max(w, 0.0))
    return out, dd * np.concatenate([W[k] * gd for k in range(n)])


# ------------------------------------------------------------------ CSG ----

def union(*sdfs):
    """Union of shapes given by distances positive outside: the minimum."""
    return np.minimum.reduce([np.asarray(s, dtype=np.float64) for s in sdfs])


def intersection(*sdfs):
    """Intersection of shapes given by distances positive outside: the maximum."""
    return np.maximum.reduce([np.asarray(s, dtype=np.float64) for s in sdfs])


# ------------------------------------------------- many points at once ----
# The same quantities as shape2d_sdf for an array of points: the roots of
# every point's quintic (and crossing cubic) are the eigenvalues of its
# companion matrix, computed for all points in one batched call.

def _batched_roots(coef):
    """Roots (M, n) of the polynomials with ascending coefficients (M, n+1)
    and a common nonzero leading coefficient."""
    n = coef.shape[1] - 1
    comp = np.zeros((coef.shape[0], n, n))
    comp[:, 1:, :-1] = np.eye(n - 1)
    comp[:, :, -1] = -coef[:, :-1] / coef[:, -1:]
    return np.linalg.eigvals(comp)


def shape2d_sdf_many(c, rho1, rho2, X, with_grad=False):
    """shape2d_sdf over points X (M, 2): distances (M,) and optionally the
    radius gradients (M, 2N)."""
    X = np.asarray(X, dtype=np.float64)
    C = control_points(c, rho1, rho2)
    N = len(C)
    M = X.shape[0]
    best_d = np.full(M, np.inf)
    best_i = np.zeros(M, dtype=int)
    best_s = np.zeros(M)
    cross = np.zeros(M, dtype=int)
    for i in range(N):
        a = _power(C[i])
        db = np.array([a[1], 2 * a[2], 3 * a[3]])
        q = np.zeros((M, 6))
        for p in range(4):
            bp = (a[p] - X) if p == 0 else np.broadcast_to(a[p], X.shape)
            for j in range(3):
                q[:, p + j] += bp @ db[j]
        cand = np.concatenate([np.zeros((M, 1)), np.ones((M, 1)), np.full((M, 5), np.nan)], axis=1)
        if abs(q[0, 5]) > 0.0:
            r = _batched_roots(q)
            ok = (np.abs(r.imag) < 1e-9) & (r.real > 0.0) & (r.real < 1.0)
            cand[:, 2:] = np.where(ok, r.real, np.nan)
        else:                               # degenerate segment: one point at a time
            for m in range(M):
                _, s = closest_on_segment(C[i], X[m])
                cand[m, 2] = s
        pts = np.einsum("mkr,rx->mkx", bernstein(np.nan_to_num(cand, nan=0.0)), C[i])
        dist = np.linalg.norm(pts - X[:, None, :], axis=-1)
        dist = np.where(np.isnan(cand), np.inf, dist)
        k = np.argmin(dist, axis=1)
        dmin = dist[np.arange(M), k]
        better = dmin < best_d
        best_d = np.where(better, dmin, best_d)
        best_i = np.where(better, i, best_i)
        best_s = np.where(better, cand[np.arange(M), k], best_s)
        # even-odd crossings of the ray towards +x
        cy = np.stack([np.full(M, a[0][1]) - X[:, 1], np.full(M, a[1][1]),
                       np.full(M, a[2][1]), np.full(M, a[3][1])], axis=1)
        if a[3][1] != 0.0:
            r = _batched_roots(cy)
            ok = (np.abs(r.imag) < 1e-12) & (r.real >= 0.0) & (r.real < 1.0)
            s = np.where(ok, r.real, 0.0)
            bx = np.einsum("mkr,r->mk", bernstein(s), C[i][:, 0])
            cross += np.sum(ok & (bx > X[:, :1]), axis=1)
        else:
            cross += np.array([_crossings(C[i], X[m]) for m in range(M)])
    inside = cross % 2 == 1
    sd = np.where(inside, -best_d, best_d)
    if not with_grad:
        return sd
    # the envelope gradient of shape2d_sdf, for all points at once
    seg = np.minimum(best_i, N - 1)
    foot = np.einsum("mr,mrx->mx", bernstein(best_s), C[seg])
    nrm = np.where(best_d[:, None] > 0.0, (X - foot) / np.where(best_d > 0.0, best_d, 1.0)[:, None], 0.0)
    base = 2.0 * np.pi * np.arange(N) / N
    ang = np.empty(2 * N)
    ang[0::2] = base + 2.0 * np.pi / (3.0 * N)
    ang[1::2] = base + 4.0 * np.pi / (3.0 * N)
    U = np.stack([np.cos(ang), np.sin(ang)], axis=-1)          # (2N, 2)
    nu = nrm @ U.T                                             # (M, 2N)
    w = bernstein(best_s)                                      # (M, 4)
    J = control_jacobian(N)
    grad = np.zeros((M, 2 * N))
    for r in range(4):
        grad -= nu * w[:, r:r + 1] * J[seg, r, :]
    grad = np.where(inside[:, None], -grad, grad)
    return sd, grad


def _controls_per_point(c, r1, r2):
    """Control polygons (M, N, 4, 2) from per-point centres (M, 2) and radii
    (M, N): the construction of control_points for every point."""
    N = r1.shape[1]
    base = 2.0 * np.pi * np.arange(N) / N
    a0 = base + 2.0 * np.pi / (3.0 * N)
    a1 = base + 4.0 * np.pi / (3.0 * N)
    p0 = c[:, None, :] + r1[..., None] * np.stack([np.cos(a0), np.sin(a0)], axis=-1)
    p1 = c[:, None, :] + r2[..., None] * np.stack([np.cos(a1), np.sin(a1)], axis=-1)
    e0 = 0.5 * (np.roll(p1, 1, axis=1) + p0)
    e1 = np.roll(e0, -1, axis=1)
    return np.stack([e0, p0, p1, e1], axis=2)


def _sdf2d_points(Cp, X, samples=24, newton=5):
    """Outside-positive distance of each point X[m] to its own closed curve
    Cp[m], with the closest segment, parameter and the inside flag.

    The closest parameter of each segment starts at the nearest of
    ``samples`` evenly spaced ones and is refined by Newton steps on
    (B - x) . B' = 0, kept in [0, 1]. The side comes from the outward normal
    at the closest point (the curve turns counter-clockwise: radii at
    increasing polar angles). This is a faster evaluation of the same
    distance as shape2d_sdf, which checks it."""
    M, N = Cp.shape[:2]
    rows = np.arange(M)
    s0 = np.linspace(0.0, 1.0, samples)
    Bs = bernstein(s0)                                          # (S, 4)
    best_d = np.full(M, np.inf)
    best_i = np.zeros(M, dtype=int)
    best_s = np.zeros(M)
    for i in range(N):
        P = Cp[:, i]                                            # (M, 4, 2)
        pts = Bs @ P                                            # (M, S, 2)
        k = np.argmin(np.sum((pts - X[:, None, :]) ** 2, axis=-1), axis=1)
        sv = s0[k]
        e0, p0, p1, e1 = (P[:, r] for r in range(4))
        for _ in range(newton):
            u = 1.0 - sv
            B = (u ** 3)[:, None] * e0 + (3 * u * u * sv)[:, None] * p0 \
                + (3 * u * sv * sv)[:, None] * p1 + (sv ** 3)[:, None] * e1
            d1 = (3 * u * u)[:, None] * (p0 - e0) + (6 * u * sv)[:, None] * (p1 - p0) \
                + (3 * sv * sv)[:, None] * (e1 - p1)
            d2 = (6 * u)[:, None] * (p1 - 2 * p0 + e0) + (6 * sv)[:, None] * (e1 - 2 * p1 + p0)
            r = B - X
            f1 = np.sum(r * d1, axis=1)
            f2 = np.sum(d1 * d1, axis=1) + np.sum(r * d2, axis=1)
            step = np.where(f2 > 0.0, f1 / np.where(f2 > 0.0, f2, 1.0), 0.0)
            sv = np.clip(sv - step, 0.0, 1.0)
        dist = np.linalg.norm((bernstein(sv)[:, None, :] @ P)[:, 0] - X, axis=1)
        better = dist < best_d
        best_d = np.where(better, dist, best_d)
        best_i = np.where(better, i, best_i)
        best_s = np.where(better, sv, best_s)
    P = Cp[rows, best_i]
    u, sv = 1.0 - best_s, best_s
    foot = np.einsum("mr,mrx->mx", bernstein(best_s), P)
    tan = (3 * u * u)[:, None] * (P[:, 1] - P[:, 0]) + (6 * u * sv)[:, None] * (P[:, 2] - P[:, 1]) \
        + (3 * sv * sv)[:, None] * (P[:, 3] - P[:, 2])
    outward = np.stack([tan[:, 1], -tan[:, 0]], axis=1)         # right of a CCW tangent
    inside = np.sum((X - foot) * outward, axis=1) < 0.0
    return np.where(inside, -best_d, best_d), best_d, best_i, best_s, inside


def extrude_sdf_many(shape, X, with_grad=False):
    """extrude_sdf over points X (M, 3): every point gets its own
    interpolated cross-section."""
    X = np.asarray(X, dtype=np.float64)
    keys = shape["keys"]
    n = len(keys)
    z0, z1 = float(shape["z0"]), float(shape["z1"])
    zm, h = 0.5 * (z0 + z1), 0.5 * (z1 - z0)
    M = X.shape[0]
    u = np.clip((X[:, 2] - z0) / (z1 - z0), 0.0, 1.0)
    if n == 1:
        W = np.ones((M, 1))
    else:
        uk = np.arange(n) / (n - 1)
        coeff = np.linalg.solve(np.vander(uk, n, increasing=True), np.eye(n))
        W = (u[:, None] ** np.arange(n)) @ coeff               # (M, n)
    kc = np.array([np.asarray(k["c"], dtype=np.float64) for k in keys])      # (n, 2)
    k1 = np.array([np.asarray(k["rho1"], dtype=np.float64) for k in keys])   # (n, N)
    k2 = np.array([np.asarray(k["rho2"], dtype=np.float64) for k in keys])
    c, r1, r2 = W @ kc, W @ k1, W @ k2
    Cp = _controls_per_point(c, r1, r2)
    d, dist, seg, sbest, inside = _sdf2d_points(Cp, X[:, :2])
    w = np.abs(X[:, 2] - zm) - h
    nrm = np.hypot(np.maximum(d, 0.0), np.maximum(w, 0.0))
    out = np.minimum(np.maximum(d, w), 0.0) + nrm
    if not with_grad:
        return out
    N = r1.shape[1]
    foot = np.einsum("mr,mrx->mx", bernstein(sbest), Cp[np.arange(M), seg])
    nv = np.where(dist[:, None] > 0.0, (X[:, :2] - foot) / np.where(dist > 0.0, dist, 1.0)[:, None], 0.0)
    base = 2.0 * np.pi * np.arange(N) / N
    ang = np.empty(2 * N)
    ang[0::2] = base + 2.0 * np.pi / (3.0 * N)
    ang[1::2] = base + 4.0 * np.pi / (3.0 * N)
    U = np.stack([np.cos(ang), np.sin(ang)], axis=-1)
    nu = nv @ U.T
    bw = bernstein(sbest)
    J = control_jacobian(N)
    g2 = np.zeros((M, 2 * N))
    for r in range(4):
        g2 -= nu * bw[:, r:r + 1] * J[seg, r, :]
    g2 = np.where(inside[:, None], -g2, g2)
    both_in = (d <= 0.0) & (w <= 0.0)
    dd = np.where(both_in, (d >= w).astype(np.float64),
                  np.maximum(d, 0.0) / np.where(nrm > 0.0, nrm, 1.0))
    grad = np.concatenate([(dd * W[:, k])[:, None] * g2 for k in range(n)], axis=1)
    return out, grad
