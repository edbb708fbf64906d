"""The verification configurations at their stated sizes, CUDA path against
the FP64 oracle.

- Config 1: translating sphere, 32^3, 20 steps, initial projection, final
  kinetic energy and its gradient with respect to the sphere's velocity v.
  The stated solver is plain FP64 CG to relative residual 1e-10; FP64 MGPCG
  and MIXED run the same rollout.
- Config 3: rotating plate, 64^3, 16 steps, 4 angle knots; the GPU adjoint
  in FP32 and MIXED (and FP64) against the oracle's adjoint and against
  central finite differences of the oracle's loss (h = 1e-4), the gradient
  check of Sec. 2.3.2-2.3.3.
- Config 4 at 64^3: one cut-cell projection of a divergent N(0, 1) velocity
  around 64 static spheres, by FP64 MGPCG, FP32 MGPCG and MIXED to 1e-8, each
  velocity against the oracle's unpreconditioned CG to 1e-12 (computed here:
  about three minutes of host time).

The oracle values of configs 1 and 3 are stored in
tests/golden/oracle_configs.json by tests/golden/make_golden.py --configs,
which calls only the oracle.
"""

import json
import os

import numpy as np
import pytest

import nf_inputs as I
from tests.test_gpu_parity import solver_warnings

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "oracle_configs.json")) as f:
    STORED = json.load(f)["cases"]

# Tolerances. MIXED and FP32: the velocity (here the loss, a quadratic of it)
# relative 1e-5 and the gradient relative 1e-4. FP64 paths are held tighter:
# the oracle solves to 1e-12, the GPU to the tolerance in the test, so their
# difference is set by the GPU solve's residual carried through the rollout.
LOSS_TOL = {"fp64": 1e-8, "mixed": 1e-5, "fp32": 1e-5}
GRAD_TOL = {"fp64": 1e-6, "mixed": 1e-4, "fp32": 1e-4}
# central differences with h = 1e-4 cross the kinks of the trilinear
# interpolation and the fraction ramp: the oracle's own adjoint and its FD
# agree to a few 1e-3 relative, and the GPU gradient is held to this band
FD_BAND = 1e-2


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _rollout(nf, cfg, prec, solver, tol, dtype=torch.float64):
    ctx = nf.Context(prec, solver, tol=tol, max_iters=20000, checkpoint_every=10)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    recording, check = solver_warnings(prec)
    with recording():
        s0 = ep.set_velocity([torch.tensor(x, device="cuda", dtype=dtype) for x in cfg["u0"]],
                             project=cfg["project_initial"])
        fs = ep.step(cfg["steps"])
        J, gU = ep.loss(cfg["loss"], want_grad=True)
        gth, _, bs = ep.backward(gU, want_gU0=False)
    check(s0, fs, bs)
    ep.close()
    ctx.close()
    return J, gth, fs


@pytest.mark.parametrize("prec,solver,tol", [("fp64", "cg", 1e-10), ("fp64", "mgpcg", 1e-12),
                                             ("mixed", "mgpcg", 1e-10)])
def test_config1_sphere32_20_steps(nf, prec, solver, tol):
    cfg = I.config_sphere(32, steps=20)
    ref = STORED["config1_sphere32_s20"]
    J, gth, fs = _rollout(nf, cfg, prec, solver, tol)
    assert fs["steps"] == 20
    assert abs(J - ref["loss"]) <= LOSS_TOL[prec] * abs(ref["loss"])
    assert _rel(gth, ref["dJ_dtheta"]) <= GRAD_TOL[prec]
    assert _rel(gth, ref["dJ_dtheta_fd"]) <= FD_BAND


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("mixed", 1e-10), ("fp64", 1e-12)])
def test_config3_plate64_16_steps_adjoint_and_fd(nf, prec, tol):
    cfg = I.config_plate(64, steps=16)
    ref = STORED["config3_plate64_s16"]
    J, gth, fs = _rollout(nf, cfg, prec, "mgpcg", tol)
    assert fs["steps"] == 16
    assert abs(J - ref["loss"]) <= LOSS_TOL[prec] * abs(ref["loss"])
    assert _rel(gth, ref["dJ_dtheta"]) <= GRAD_TOL[prec]
    assert _rel(gth, ref["dJ_dtheta_fd"]) <= FD_BAND


@pytest.fixture(scope="module")
def spheres64_oracle():
    from oracle import Grid, project
    from oracle import step as S
    cfg = I.config_spheres(64)
    g = Grid(cfg["grid"])
    alpha, us = S.geometry_at(g, cfg["scene"], 0.0)
    U, _, info = project.project(g, alpha, us, cfg["u0"], 1e-12)
    assert info["rel_residual"] <= 1e-12
    return cfg, U


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_config4_spheres64_projection_against_oracle(nf, spheres64_oracle, prec):
    cfg, U_ref = spheres64_oracle
    ctx = nf.Context(prec, "mgpcg", tol=1e-8, max_iters=5000)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    recording, check = solver_warnings(prec)
    with recording():
        st = ep.set_velocity([torch.tensor(x, device="cuda") for x in cfg["u0"]], project=True)
    # FP32 without refinement stalls above 1e-8 (the finding the precision
    # sweep reports); FP64 and MIXED reach it
    if prec != "fp32":
        check(st)
        assert st["rel_residual"] <= 1e-8
    else:
        assert st["rel_residual"] <= 1e-5
    got = [t.cpu().numpy() for t in ep.velocity()]
    ep.close()
    ctx.close()
    err = _rel(np.concatenate([x.ravel() for x in got]),
               np.concatenate([x.ravel() for x in U_ref]))
    assert err <= {"fp64": 1e-7, "fp32": 1e-5, "mixed": 1e-5}[prec]
