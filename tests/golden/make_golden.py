"""Write the stored oracle values in this folder (calls only ``oracle/``).

Run from the repository root: ``python tests/golden/make_golden.py`` (the
small cases, ``oracle_small.json``) or ``... --configs`` (the verification
configurations at their stated sizes, ``oracle_configs.json``). The
values are the FP64 oracle's loss and parameter gradient of small seeded
rollouts (the sphere, chamber and plate scenes of the workload generator at
reduced size). The paper
prints no worked numeric example for this path, so no stored value here is
the paper's; these guard the oracle against unintended change, and any
regeneration must name, in its commit message, the passage that justifies
the change of the oracle's arithmetic.
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import nf_inputs as I  # noqa: E402
from oracle import step as S  # noqa: E402

CASES = {
    "sphere12_s2": lambda: I.config_sphere(12, steps=2),
    "plate12_s2": lambda: I.config_plate(12, steps=2),
    "chamber16_s3": lambda: I.config_chamber(16, steps=3, duct_half_cells=2),
    "chamber16_s3_cfl1": lambda: I.config_chamber(16, steps=3, duct_half_cells=2, cfl_max=1.0),
}


def _viscous_sphere():
    cfg = I.config_sphere(12, steps=2)
    cfg["grid"]["nu"] = 0.05                       # Eq. viscosity_matrix
    return cfg


def _corner_plate():
    cfg = I.config_plate(12, steps=2)
    cfg["grid"]["fractions"] = "corner"            # Sec. 2.3.1, face-area fractions
    return cfg


def _extruded_obstacles():
    g = I.make_grid(10, 0.01)
    g["fractions"] = "corner"
    return dict(name="extruded10", grid=g, scene=I.extruded_scene(4, shapes=2, keys=2),
                u0=I.gaussian_faces(g, 0.1, 21), project_initial=True, steps=2, tol=1e-12,
                loss="kinetic_energy")               # App. A shapes


# options the oracle has beyond the cases the CUDA path is also held to here
ORACLE_CASES = {
    "sphere12_s2_viscous": _viscous_sphere,
    "plate12_s2_corner": _corner_plate,
    "extruded10_s2_corner": _extruded_obstacles,
}


# The verification configurations at their stated sizes (the workload
# generator's configs 1 and 3): the FP64 oracle's loss, its adjoint dJ/dtheta
# and central finite differences of J with step h = 1e-4 (the gradient check
# of Sec. 2.3.2-2.3.3). Every CG solve goes to relative residual 1e-12.
CONFIG_CASES = {
    "config1_sphere32_s20": lambda: I.config_sphere(32, steps=20),
    "config3_plate64_s16": lambda: I.config_plate(64, steps=16),
}
CONFIG_TOL = 1e-12
CONFIG_FD_H = 1e-4


def _config_job(job):
    """One unit of work: ('adjoint', name) or ('loss', name, k, sign)."""
    import numpy as np
    name = job[1]
    cfg = CONFIG_CASES[name]()
    if job[0] == "adjoint":
        J, gth, info = S.loss_and_grad(cfg, tol=CONFIG_TOL)
        its = [t["iters"] for t in info["tapes"]]
        return job, {"loss": J, "dJ_dtheta": [float(x) for x in gth],
                     "steps": len(info["tapes"]), "max_cg_iters": int(max(its))}
    _, _, k, sign = job
    th = np.asarray(cfg["scene"]["theta"], dtype=np.float64)
    th[k] += sign * CONFIG_FD_H
    return job, S.loss_only(cfg, th, tol=CONFIG_TOL)


def compute_configs(procs=None):
    """The stored values of CONFIG_CASES, the jobs spread over processes."""
    import multiprocessing as mp
    jobs = []
    for name, make in CONFIG_CASES.items():
        K = len(make()["scene"]["theta"])
        jobs.append(("adjoint", name))
        jobs += [("loss", name, k, sgn) for k in range(K) for sgn in (1, -1)]
    with mp.get_context("spawn").Pool(procs or min(len(jobs), os.cpu_count() or 1)) as pool:
        res = dict(pool.map(_config_job, jobs))
    out = {}
    for name, make in CONFIG_CASES.items():
        K = len(make()["scene"]["theta"])
        o = dict(res[("adjoint", name)])
        o["fd_h"] = CONFIG_FD_H
        o["dJ_dtheta_fd"] = [(res[("loss", name, k, 1)] - res[("loss", name, k, -1)]) /
                             (2 * CONFIG_FD_H) for k in range(K)]
        out[name] = o
    return out


def compute(name):
    cfg = (CASES.get(name) or ORACLE_CASES[name])()
    J, gth, info = S.loss_and_grad(cfg, tol=1e-13)
    return {"loss": J, "dJ_dtheta": [float(x) for x in gth], "steps": len(info["tapes"])}


def main():
    if "--configs" in sys.argv:
        # about half an hour of CPU time, spread over the host's cores
        out = {"generator": "tests/golden/make_golden.py --configs", "tol": CONFIG_TOL,
               "cases": compute_configs()}
        with open(os.path.join(HERE, "oracle_configs.json"), "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        return
    out = {"generator": "tests/golden/make_golden.py", "tol": 1e-13,
           "cases": {k: compute(k) for k in list(CASES) + list(ORACLE_CASES)}}
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
