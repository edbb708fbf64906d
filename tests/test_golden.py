"""Stored oracle values (tests/golden/oracle_small.json).

CPU: the oracle still produces them (guards its arithmetic against
unintended change). GPU: the CUDA path matches them in every precision mode
(FP64 to 1e-8, FP32 and MIXED to the 1e-4 gradient bar).
"""

import json
import os

import numpy as np
import pytest

from tests.golden.make_golden import CASES, ORACLE_CASES, compute
from tests.test_gpu_parity import solver_warnings

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "oracle_small.json")) as f:
    GOLDEN = json.load(f)["cases"]


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("name", sorted(CASES) + sorted(ORACLE_CASES))
def test_oracle_reproduces_stored_values(name):
    got = compute(name)
    ref = GOLDEN[name]
    assert got["steps"] == ref["steps"]
    assert abs(got["loss"] - ref["loss"]) <= 1e-9 * abs(ref["loss"])
    assert _rel(got["dJ_dtheta"], ref["dJ_dtheta"]) <= 1e-8


@pytest.mark.gpu
@pytest.mark.parametrize("prec,jtol,gtol", [("fp64", 1e-9, 1e-8), ("mixed", 1e-5, 1e-4),
                                            ("fp32", 1e-5, 1e-4)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_cuda_path_matches_stored_values(nf, name, prec, jtol, gtol):
    import torch
    cfg = CASES[name]()
    ref = GOLDEN[name]
    ctx = nf.Context(prec, "mgpcg", tol={"fp64": 1e-12, "mixed": 1e-10, "fp32": 1e-6}[prec],
                     max_iters=3000, checkpoint_every=2, cfl_max=cfg.get("cfl_max", 0.0))
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    recording, check = solver_warnings(prec)
    with recording():
        s0 = ep.set_velocity([torch.tensor(x, device="cuda", dtype=torch.float64)
                              for x in cfg["u0"]], project=cfg["project_initial"])
        st = ep.step(cfg["steps"])
        J, gU = ep.loss(cfg["loss"], want_grad=True)
        gth, _, bs = ep.backward(gU)
    check(s0, st, bs)
    ep.close()
    ctx.close()
    assert st["steps"] + int(cfg["project_initial"]) == ref["steps"]
    assert abs(J - ref["loss"]) <= jtol * abs(ref["loss"])
    assert _rel(gth, ref["dJ_dtheta"]) <= gtol


# The verification configurations at their stated sizes (stored by
# make_golden.py --configs, about 20 minutes of host time): the oracle's own
# adjoint agrees with central differences of its loss (h = 1e-4) within the
# band set by the kinks of trilinear interpolation and the fraction ramp
with open(os.path.join(HERE, "golden", "oracle_configs.json")) as f:
    CONFIGS_STORED = json.load(f)["cases"]


@pytest.mark.parametrize("name,band", [("config1_sphere32_s20", 1e-3),
                                       ("config3_plate64_s16", 1e-2)])
def test_stored_config_adjoint_matches_its_central_differences(name, band):
    ref = CONFIGS_STORED[name]
    assert _rel(ref["dJ_dtheta"], ref["dJ_dtheta_fd"]) <= band
    assert ref["fd_h"] == 1e-4
