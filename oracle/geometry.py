"""Analytic solid geometry of the FP64 oracle (test infrastructure only).

Sec. 2.3.1 (Projection) takes the solid's signed distance ``phi`` and velocity
``u_s`` at t_{n+1} from the geometry; Sec. 2.3.3 chains the gradient through
them to the parameters. Sign convention: ``phi > 0`` in the fluid, ``phi < 0``
in the solid. Union of solid-complement pieces is ``max`` of their ``phi``
(the CSG union of Sec. 2.2 acting on fluid regions).

Every function takes physical positions ``x`` of shape ``(..., 3)`` (x, y, z)
and a time ``t`` and returns:

* ``phi(scene, x, t)``            -> ``(...)``
* ``solid_velocity(scene, x, t)`` -> ``(..., 3)``
* ``dphi_dtheta(scene, x, t)``    -> ``(..., K)``
* ``dus_dtheta(scene, x, t)``     -> ``(..., 3, K)``
"""

from __future__ import annotations

import numpy as np

from . import bezier

FAR = 1.0e3   # phi of a scene without solid: every ramp sample saturates to 1


def n_params(scene):
    return len(scene.get("theta", []))


# ------------------------------------------------------------ box SDF -----

def box_sdf(p, h):
    """Exact signed distance to the box ``|p_a| <= h_a`` (positive outside)."""
    q = np.abs(p) - np.asarray(h)
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(np.max(q, axis=-1), 0.0)
    return outside + inside


def box_sdf_grad(p, h):
    """Gradient of :func:`box_sdf` with respect to ``p``."""
    q = np.abs(p) - np.asarray(h)
    sgn = np.where(p >= 0.0, 1.0, -1.0)
    m = np.maximum(q, 0.0)
    nm = np.linalg.norm(m, axis=-1, keepdims=True)
    out_grad = sgn * m / np.where(nm > 0.0, nm, 1.0)
    a = np.argmax(q, axis=-1)
    in_grad = np.zeros_like(p)
    np.put_along_axis(in_grad, a[..., None],
                      np.take_along_axis(sgn, a[..., None], axis=-1), axis=-1)
    is_out = (nm[..., 0] > 0.0)[..., None]
    return np.where(is_out, out_grad, in_grad)


# ---------------------------------------------------- time dependences -----

def chamber_radius(scene, t):
    """Radius modulation s(t), its rate and their theta-derivatives."""
    th = np.asarray(scene["theta"])
    a, b = th[:4], th[4:]
    k = np.arange(1, 5)
    w = 2.0 * np.pi * k / scene["period"]
    cs, sn = np.cos(w * t), np.sin(w * t)
    s = 1.0 + np.sum(a * cs + b * sn)
    sdot = np.sum(w * (-a * sn + b * cs))
    ds = np.concatenate([cs, sn])
    dsdot = np.concatenate([-w * sn, w * cs])
    return s, sdot, ds, dsdot


def plate_angle(scene, t):
    """Piecewise-linear angle through 4 knots at t = 0, T/3, 2T/3, T.

    Returns the angle, its rate, and their theta-derivatives.
    """
    th = np.asarray(scene["theta"])
    seg_len = scene["period"] / 3.0
    seg = int(min(max(np.floor(t / seg_len), 0), 2))
    tau = (t - seg * seg_len) / seg_len
    ang = th[seg] * (1.0 - tau) + th[seg + 1] * tau
    omega = (th[seg + 1] - th[seg]) / seg_len
    dang = np.zeros(4)
    dang[seg], dang[seg + 1] = 1.0 - tau, tau
    domega = np.zeros(4)
    domega[seg], domega[seg + 1] = -1.0 / seg_len, 1.0 / seg_len
    return ang, omega, dang, domega


def _plate_local(scene, x, ang):
    c = np.asarray(scene["centre"])
    r = x - c
    ca, sa = np.cos(ang), np.sin(ang)
    p = np.stack([ca * r[..., 0] + sa * r[..., 1],
                  -sa * r[..., 0] + ca * r[..., 1],
                  r[..., 2]], axis=-1)
    return p, r


def _chamber_parts(scene, x, t):
    c0 = np.asarray(scene["centre"])
    ax = np.asarray(scene["axes"])
    s, sdot, ds, dsdot = chamber_radius(scene, t)
    rho = np.linalg.norm((x - c0) / ax, axis=-1)
    phi_ell = ax.min() * (s - rho)
    x0 = scene["duct_x0"]
    hw = scene["duct_half"]
    dc = np.array([(x0 + 2.0) / 2.0, c0[1], c0[2]])
    dh = np.array([(2.0 - x0) / 2.0, hw, hw])
    phi_duct = -box_sdf(x - dc, dh)
    ell = phi_ell >= phi_duct
    return phi_ell, phi_duct, ell, (s, sdot, ds, dsdot)


def _shell_parts(scene, x, t):
    v = np.asarray(scene["theta"])
    lo = np.asarray(scene["lo"]) + v * t
    hi = np.asarray(scene["hi"]) + v * t
    th = scene["thickness"]
    c = 0.5 * (lo + hi)
    h_out = 0.5 * (hi - lo)
    h_in = h_out - th
    return x - c, h_out, h_in


def pulse_scale(scene, t):
    """Contraction of an ``extruded`` scene's pulsing shape: the factor k(t)
    applied to its radii, piecewise linear through 4 knots (theta) at
    t = 0, T/3, 2T/3, T; returns k, its rate and their theta-derivatives."""
    th = np.asarray(scene["theta"], dtype=np.float64)
    seg_len = scene["pulse"]["period"] / 3.0
    seg = int(min(max(np.floor(t / seg_len), 0), 2))
    tau = (t - seg * seg_len) / seg_len
    k = th[seg] * (1.0 - tau) + th[seg + 1] * tau
    kdot = (th[seg + 1] - th[seg]) / seg_len
    dk = np.zeros(4)
    dk[seg], dk[seg + 1] = 1.0 - tau, tau
    dkdot = np.zeros(4)
    dkdot[seg], dkdot[seg + 1] = -1.0 / seg_len, 1.0 / seg_len
    return k, kdot, dk, dkdot


def _extruded_radii(scene):
    """Base radii (2N,) of every key of every shape: theta when the radii are
    the parameters (``params = "radii"``, the default), else the keys' own."""
    th = np.asarray(scene["theta"], dtype=np.float64)
    from_theta = scene.get("params", "radii") == "radii"
    out, j = [], 0
    for sh in scene["shapes"]:
        rs = []
        for k in sh["keys"]:
            n2 = 2 * int(k["nseg"])
            if from_theta:
                rs.append(th[j:j + n2])
                j += n2
            else:
                rs.append(np.asarray(k["rho"], dtype=np.float64))
        out.append(rs)
    return out


def _local(sh, Xw):
    """Points in the shape's frame, and the frame's axes (rows: local x, y, z
    in world coordinates)."""
    fr = sh.get("frame")
    if fr is None:
        return Xw, np.eye(3)
    A = np.asarray(fr["axes"], dtype=np.float64)
    return (Xw - np.asarray(fr["origin"], dtype=np.float64)) @ A.T, A


def _extruded(scene, x, t, with_grad):
    """Outside-positive distance to each shape of an ``extruded`` scene and,
    with ``with_grad``, its theta-gradient (M, K).

    Shapes: ``dict(z0, z1, keys=[dict(c, nseg[, rho])...][, frame])``. A shape
    with a rigid frame ``dict(origin, axes)`` (axes orthonormal, rows the
    local x, y, z in world coordinates) is extruded along its local z and a
    world point x is measured at axes (x - origin), which keeps distances.
    theta is either every radius, shape by shape, key by key (rho1_0, rho2_0,
    rho1_1, ...), or, with ``params = "pulse"``, the 4 knots of the
    contraction k(t) of shape ``pulse["shape"]``, whose radii are k(t) times
    its keys' own."""
    Xw = x.reshape(-1, 3)
    radii = _extruded_radii(scene)
    pulse = scene.get("pulse")
    kt = pulse_scale(scene, t) if pulse else None
    K = len(scene["theta"])
    dists, grads, j = [], [], 0
    for s_, sh in enumerate(scene["shapes"]):
        X, _ = _local(sh, Xw)
        scale = kt[0] if (pulse and s_ == pulse["shape"]) else 1.0
        keys = [dict(c=k["c"], rho1=scale * r[0::2], rho2=scale * r[1::2])
                for k, r in zip(sh["keys"], radii[s_])]
        shape = dict(z0=sh["z0"], z1=sh["z1"], keys=keys)
        if not with_grad:
            dists.append(bezier.extrude_sdf_many(shape, X))
            continue
        d, g = bezier.extrude_sdf_many(shape, X, with_grad=True)
        G = np.zeros((X.shape[0], K))
        if scene.get("params", "radii") == "radii":
            G[:, j:j + g.shape[1]] = scale * g
            j += g.shape[1]
        elif pulse and s_ == pulse["shape"]:
            # d d / d k = sum over the scaled radii of g times the base radius
            G[:, :] = (g @ np.concatenate(radii[s_]))[:, None] * kt[2][None, :]
        dists.append(d)
        grads.append(G)
    return dists, grads


def _extruded_phi(scene, x, t, with_grad=False):
    """phi > 0 in the fluid: outside the union of the shapes (obstacles) or
    inside it (containers): CSG union is the min of the distances."""
    dists, grads = _extruded(scene, x, t, with_grad)
    D = np.stack(dists)                                   # (shapes, M)
    a = np.argmin(D, axis=0)
    sgn = 1.0 if scene["fluid"] == "outside" else -1.0
    rows = np.arange(D.shape[1])
    ph = sgn * D[a, rows]
    if not with_grad:
        return ph.reshape(x.shape[:-1])
    G = sgn * np.stack(grads)[a, rows]                    # (M, K)
    K = len(scene["theta"])
    return ph.reshape(x.shape[:-1]), G.reshape(x.shape[:-1] + (K,))


def _extruded_us(scene, x, t, with_grad=False):
    """Solid velocity: where the pulsing shape is the nearest (the active
    piece of the union), the velocity of its uniform contraction about the
    cross-section centre, (kdot / k) (p - c(z)) across its local z; zero
    elsewhere and on static scenes. With ``with_grad`` also d u_s / d theta."""
    Xw = x.reshape(-1, 3)
    K = len(scene["theta"])
    out = np.zeros(Xw.shape)
    dout = np.zeros(Xw.shape + (K,))
    pulse = scene.get("pulse")
    if pulse:
        dists, _ = _extruded(scene, x, t, False)
        act = np.argmin(np.stack(dists), axis=0) == pulse["shape"]
        sh = scene["shapes"][pulse["shape"]]
        X, A = _local(sh, Xw)
        n = len(sh["keys"])
        z0, z1 = float(sh["z0"]), float(sh["z1"])
        u = np.clip((X[:, 2] - z0) / (z1 - z0), 0.0, 1.0)
        W = np.stack([bezier.lagrange_weights(n, uu) for uu in u])      # (M, n)
        c = W @ np.array([np.asarray(k["c"], dtype=np.float64) for k in sh["keys"]])
        r = np.zeros(Xw.shape)
        r[:, :2] = X[:, :2] - c
        dirw = np.where(act[:, None], r @ A, 0.0)          # back to world axes
        k, kdot, dk, dkdot = pulse_scale(scene, t)
        out = (kdot / k) * dirw
        coef = (dkdot * k - kdot * dk) / (k * k)          # d(kdot / k) / d theta
        dout = dirw[..., None] * coef
    if with_grad:
        return out.reshape(x.shape), dout.reshape(x.shape + (K,))
    return out.reshape(x.shape)


# ------------------------------------------------------------ dispatch -----

def phi(scene, x, t):
    kind = scene["kind"]
    if kind == "none":
        return np.full(x.shape[:-1], FAR)
    if kind == "sphere":
        c = np.asarray(scene["centre"]) + np.asarray(scene["theta"]) * t
        return np.linalg.norm(x - c, axis=-1) - scene["radius"]
    if kind == "spheres":
        out = np.full(x.shape[:-1], FAR)
        for cx, cy, cz, r in scene["spheres"]:
            d = np.linalg.norm(x - np.array([cx, cy, cz]), axis=-1) - r
            out = np.minimum(out, d)
        return out
    if kind == "chamber":
        pe, pd, _, _ = _chamber_parts(scene, x, t)
        return np.maximum(pe, pd)
    if kind == "plate":
        ang, _, _, _ = plate_angle(scene, t)
        p, _ = _plate_local(scene, x, ang)
        return box_sdf(p, scene["half"])
    if kind == "shell":
        p, ho, hi = _shell_parts(scene, x, t)
        return np.maximum(box_sdf(p, ho), -box_sdf(p, hi))
    if kind == "extruded":
        return _extruded_phi(scene, x, t)
    raise ValueError(kind)


def solid_velocity(scene, x, t):
    kind = scene["kind"]
    out = np.zeros(x.shape)
    if kind in ("sphere", "shell"):
        out[...] = np.asarray(scene["theta"])
    elif kind == "chamber":
        _, _, ell, (s, sdot, _, _) = _chamber_parts(scene, x, t)
        c0 = np.asarray(scene["centre"])
        out = np.where(ell[..., None], (sdot / s) * (x - c0), 0.0)
    elif kind == "plate":
        _, omega, _, _ = plate_angle(scene, t)
        r = x - np.asarray(scene["centre"])
        out[..., 0] = -omega * r[..., 1]
        out[..., 1] = omega * r[..., 0]
    elif kind == "extruded":
        out = _extruded_us(scene, x, t)
    return out


def dphi_dtheta(scene, x, t):
    kind = scene["kind"]
    K = n_params(scene)
    if kind in ("none", "spheres") or K == 0:
        return np.zeros(x.shape[:-1] + (K,))
    if kind == "sphere":
        c = np.asarray(scene["centre"]) + np.asarray(scene["theta"]) * t
        r = x - c
        nr = np.linalg.norm(r, axis=-1, keepdims=True)
        return -t * r / np.where(nr > 0.0, nr, 1.0)
    if kind == "chamber":
        _, _, ell, (_, _, ds, _) = _chamber_parts(scene, x, t)
        amin = np.min(scene["axes"])
        return np.where(ell[..., None], amin * ds, 0.0)
    if kind == "plate":
        ang, _, dang, _ = plate_angle(scene, t)
        p, _ = _plate_local(scene, x, ang)
        gp = box_sdf_grad(p, scene["half"])
        dphi_dang = gp[..., 0] * p[..., 1] - gp[..., 1] * p[..., 0]
        return dphi_dang[..., None] * dang
    if kind == "shell":
        p, ho, hi = _shell_parts(scene, x, t)
        so, si = box_sdf(p, ho), -box_sdf(p, hi)
        g = np.where((so >= si)[..., None], box_sdf_grad(p, ho),
                     -box_sdf_grad(p, hi))
        return -t * g
    if kind == "extruded":
        return _extruded_phi(scene, x, t, with_grad=True)[1]
    raise ValueError(kind)


def dus_dtheta(scene, x, t):
    kind = scene["kind"]
    K = n_params(scene)
    out = np.zeros(x.shape + (K,))
    if kind in ("sphere", "shell"):
        for a in range(3):
            out[..., a, a] = 1.0
    elif kind == "chamber":
        _, _, ell, (s, sdot, ds, dsdot) = _chamber_parts(scene, x, t)
        c0 = np.asarray(scene["centre"])
        coef = (dsdot * s - sdot * ds) / (s * s)              # (K,)
        val = (x - c0)[..., :, None] * coef                   # (..., 3, K)
        out = np.where(ell[..., None, None], val, 0.0)
    elif kind == "plate":
        _, _, _, domega = plate_angle(scene, t)
        r = x - np.asarray(scene["centre"])
        out[..., 0, :] = -r[..., 1:2] * domega
        out[..., 1, :] = r[..., 0:1] * domega
    elif kind == "extruded":
        out = _extruded_us(scene, x, t, with_grad=True)[1]
    return out
