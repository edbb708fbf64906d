"""One time step, rollouts, losses and back-propagation through time (oracle).

Sec. 2.3.1: a step is advection, viscosity, then projection with the
geometry evaluated at t_{n+1} = (n + 1) dt. Sec. 2.3.2: back-propagation
mirrors the forward in reverse order; Sec. 2.3.3 chains the fraction and
solid-velocity gradients into the shape and control parameters:

    dJ/dtheta += sum_f gS_f d alpha_f/d theta + gU_s,f d u_s,f/d theta.

An optional initial projection (the seeded noise made divergence free with
the t = 0 cut-cell system) is part of the rollout and of its adjoint.
Every forward quantity the adjoint needs is kept (no checkpointing here).

Sub-stepping (Sec. 3, Table 1 caption: steps are taken under the CFL
condition, so more steps are simulated than frames): with ``cfl_max > 0`` a
rollout advances frames of length dt, each split into
``m = ceil(max|U| dt / (dx cfl_max))`` equal steps, max|U| taken over all
faces at the start of the frame; step k of frame f ends at
``t = (f m + k + 1) dt / m``.
"""

from __future__ import annotations

import numpy as np

from . import advect as adv
from . import project as prj
from . import rasterize as ras
from .mac import Grid, outlet_face_mask


def geometry_at(g: Grid, scene, t, with_grad=False):
    if with_grad:
        alpha, dalpha = ras.fractions(g, scene, t, with_grad=True)
        us, dus = ras.face_solid_velocity(g, scene, t, with_grad=True)
        return alpha, us, dalpha, dus
    return ras.fractions(g, scene, t), ras.face_solid_velocity(g, scene, t)


def step(g: Grid, scene, U, n, tol, order=2, velocity_rule="blend", t1=None):
    """Advance ``U^n`` by one step of length ``g.dt`` ending at ``t1``
    (default ``(n + 1) dt``); returns the new field and a tape."""
    if t1 is None:
        t1 = (n + 1) * g.dt
    alpha, us = geometry_at(g, scene, t1)
    Ut = adv.advect(g, U, order)
    Uh = adv.viscosity(g, Ut)
    Unew, P, info = prj.project(g, alpha, us, Uh, tol, velocity_rule)
    tape = dict(kind="step", t=t1, U=U, Uh=Uh, P=P, alpha=alpha, us=us,
                system=info["system"], iters=info["iters"],
                rel_residual=info["rel_residual"], order=order, grid=g)
    return Unew, tape


def initial_projection(g: Grid, scene, U0, tol):
    alpha, us = geometry_at(g, scene, 0.0)
    U, P, info = prj.project(g, alpha, us, U0, tol)
    tape = dict(kind="project", t=0.0, U=U0, Uh=U0, P=P, alpha=alpha, us=us,
                system=info["system"], iters=info["iters"],
                rel_residual=info["rel_residual"], grid=g)
    return U, tape


def substeps(g: Grid, U, cfl_max):
    """Number of equal steps of a frame under the CFL rule."""
    if not cfl_max:
        return 1
    umax = max(float(np.max(np.abs(u))) for u in U)
    return max(1, int(np.ceil(umax * g.dt / (g.dx * cfl_max))))


def rollout(g: Grid, scene, U0, nsteps, tol, project_initial=True, order=2,
            cfl_max=0.0):
    """``nsteps`` steps (or frames, with ``cfl_max > 0``) from ``U0``."""
    tapes = []
    U = [u.copy() for u in U0]
    if project_initial:
        U, tape = initial_projection(g, scene, U, tol)
        tapes.append(tape)
    for f in range(nsteps):
        m = substeps(g, U, cfl_max)
        gs = g.with_dt(g.dt / m)
        for k in range(m):
            t1 = (f * m + k + 1) * gs.dt
            U, tape = step(gs, scene, U, None, tol, order, t1=t1)
            tapes.append(tape)
    return U, tapes


def _theta_terms(g: Grid, scene, tape, gS, gUs):
    _, _, dalpha, dus = geometry_at(tape["grid"], scene, tape["t"], with_grad=True)
    K = len(scene.get("theta", []))
    gth = np.zeros(K)
    for d in range(3):
        gth += np.tensordot(gS[d], dalpha[d], axes=gS[d].ndim)
        gth += np.tensordot(gUs[d], dus[d], axes=gUs[d].ndim)
    return gth


def step_adjoint(g: Grid, scene, tape, gU, tol):
    """Map ``dJ/dU^{n+1}`` to ``dJ/dU^n`` and this step's ``dJ/dtheta``."""
    gs = tape["grid"]
    gUh, gS, gUs, y, info = prj.project_adjoint(
        gs, tape["alpha"], tape["us"], tape["Uh"], tape["P"], gU, tol,
        system=tape["system"])
    gth = _theta_terms(gs, scene, tape, gS, gUs)
    if tape["kind"] == "project":
        return gUh, gth
    gUt = adv.viscosity_adjoint(gs, gUh)
    gUn = adv.advect_adjoint(gs, tape["U"], gUt, tape["order"])
    return gUn, gth


def rollout_backward(g: Grid, scene, tapes, gU_final, tol):
    gU = [x.copy() for x in gU_final]
    K = len(scene.get("theta", []))
    gth = np.zeros(K)
    for tape in reversed(tapes):
        gU, gt = step_adjoint(g, scene, tape, gU, tol)
        gth += gt
    return gU, gth


# --------------------------------------------------------------- losses ----

def kinetic_energy(g: Grid, U):
    """J = 1/2 sum_faces u^2 dx^3 and dJ/dU."""
    v = g.dx ** 3
    J = 0.5 * v * sum(float(np.sum(u * u)) for u in U)
    return J, [v * u for u in U]


def outflow(g: Grid, U):
    """Net flux out through the outlet patch: sum u_x dx^2 (side-signed)."""
    m = outlet_face_mask(g, 0)
    sgn = float(g.outlet["side"]) if g.outlet else 0.0
    a = g.dx * g.dx
    J = sgn * a * float(np.sum(U[0][m]))
    gU = [np.zeros_like(u) for u in U]
    gU[0][m] = sgn * a
    return J, gU


LOSSES = {"kinetic_energy": kinetic_energy, "outflow": outflow}


def loss_and_grad(cfg, theta=None, tol=None):
    """Full rollout of a config, its loss, and dJ/dtheta by the adjoint."""
    g = Grid(cfg["grid"])
    scene = dict(cfg["scene"])
    if theta is not None:
        scene["theta"] = list(theta)
    tol = cfg["tol"] if tol is None else tol
    U, tapes = rollout(g, scene, cfg["u0"], cfg["steps"], tol, cfg["project_initial"],
                       cfl_max=cfg.get("cfl_max", 0.0))
    J, gU = LOSSES[cfg["loss"]](g, U)
    gU0, gth = rollout_backward(g, scene, tapes, gU, tol)
    return J, gth, dict(U=U, tapes=tapes, gU0=gU0)


def loss_only(cfg, theta, tol=None):
    g = Grid(cfg["grid"])
    scene = dict(cfg["scene"])
    scene["theta"] = list(theta)
    tol = cfg["tol"] if tol is None else tol
    U, _ = rollout(g, scene, cfg["u0"], cfg["steps"], tol, cfg["project_initial"],
                   cfl_max=cfg.get("cfl_max", 0.0))
    return LOSSES[cfg["loss"]](g, U)[0]


def fd_gradient(cfg, h=1e-4, tol=None, which=None):
    """Central finite differences of the rollout loss w.r.t. theta."""
    theta = np.asarray(cfg["scene"]["theta"], dtype=np.float64)
    idx = range(len(theta)) if which is None else which
    out = np.zeros(len(theta))
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        out[k] = (loss_only(cfg, tp, tol) - loss_only(cfg, tm, tol)) / (2.0 * h)
    return out
