"""Parity at the full workload size: the pulsing chamber at 128^3 in the
launch configuration the benchmark times (MIXED MGPCG to 1e-6, CFL
sub-stepping with cfl_max 8, checkpoints every 10 steps, 100 frames).

The FP64 oracle cannot run this rollout in test time, so the checks are
(1) element-wise: the first frame's fractions against the oracle's
rasteriser at 128^3; (2) closed form at any size: with one opening,
incompressibility makes the final outflow equal the geometric volume rate
(a function of the final fractions and the solid velocity alone), and
dJ/dtheta its derivative (Sec. 2.3.3 chain rule through u_s with the active
set fixed). Tolerances: velocity functional 1e-5, gradient 1e-4 relative.
"""

import numpy as np
import pytest

import nf_inputs as I
from oracle import Grid, mac, project, rasterize

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FRAC_TOL = 1e-6


def _grounded_boundary_flux(g, alpha, us):
    """sum over faces with exactly one neighbour in an outlet-connected
    fluid component (outlet faces excluded) of (a_high - a_low) u_s. Such a
    face has alpha = 0, so U = u_s there, and summing G^T U = 0 over the
    grounded cells leaves the outflow equal to this flux. Floating pockets
    are left out: the gauge makes their right-hand side zero-mean, so their
    own boundary flux does not vanish for a pulsing (divergent) u_s."""
    act = project.active_cells(g, alpha)
    labels, grounded = project.components(g, alpha, act)
    keep = np.zeros_like(act)
    for lab, gr in grounded.items():
        if gr:
            keep |= labels == lab
    tot = 0.0
    for d in range(3):
        ax = mac.axis_of(d)
        pad = [(0, 0)] * 3
        pad[ax] = (1, 1)
        a = np.pad(keep, pad).astype(np.float64)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        sgn = a[tuple(hi)] - a[tuple(lo)]
        sgn[mac.outlet_face_mask(g, d)] = 0.0
        tot += float(np.sum(sgn * us[d]))
    return tot


def test_chamber_128_bench_configuration(nf):
    cfg = I.config_chamber(128, steps=100, seed=0)
    g = Grid(cfg["grid"])
    ctx = nf.Context("mixed", "mgpcg", tol=1e-6, max_iters=1000, checkpoint_every=10,
                     cfl_max=cfg["cfl_max"])
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    u0 = [torch.zeros(s, dtype=torch.float32, device="cuda") for s in ep.face_shapes]
    ep.set_velocity(u0, project=False)

    # (1) first frame: zero velocity, so one step ending at t = dt
    st1 = ep.step(1)
    assert st1["steps"] == 1
    a_gpu = [a.cpu().numpy() for a in ep.fractions()]
    a_ref = rasterize.fractions(g, cfg["scene"], g.dt)
    for d in range(3):
        err = np.abs(a_gpu[d] - a_ref[d]).max()
        assert err <= FRAC_TOL, (d, err)

    # (2) the rest of the rollout, the loss and the full adjoint
    st = ep.step(cfg["steps"] - 1)
    assert st["steps"] >= cfg["steps"] - 1
    J, gU = ep.loss("outflow", want_grad=True)
    alpha = [a.cpu().numpy() for a in ep.fractions()]   # at t = frames * dt
    gth, _, bs = ep.backward(gU, want_gU0=False)
    ep.close()
    ctx.close()
    assert bs["rel_residual"] <= 1e-6

    t = cfg["steps"] * g.dt
    us, dus = rasterize.face_solid_velocity(g, cfg["scene"], t, with_grad=True)
    geo = g.dx ** 2 * _grounded_boundary_flux(g, alpha, us)
    assert abs(J - geo) <= 1e-5 * abs(geo), (J, geo)
    K = len(cfg["scene"]["theta"])
    g_geo = np.array([g.dx ** 2 * _grounded_boundary_flux(g, alpha, [dus[d][..., k] for d in range(3)])
                      for k in range(K)])
    err = np.linalg.norm(np.asarray(gth) - g_geo) / np.linalg.norm(g_geo)
    assert err <= 1e-4, (gth, g_geo)
