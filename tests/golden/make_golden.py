"""Write the stored oracle values in this folder (calls only ``oracle/``).

Run from the repository root: ``python tests/golden/make_golden.py``. The
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


def compute(name):
    cfg = (CASES.get(name) or ORACLE_CASES[name])()
    J, gth, info = S.loss_and_grad(cfg, tol=1e-13)
    return {"loss": J, "dJ_dtheta": [float(x) for x in gth], "steps": len(info["tapes"])}


def main():
    out = {"generator": "tests/golden/make_golden.py", "tol": 1e-13,
           "cases": {k: compute(k) for k in list(CASES) + list(ORACLE_CASES)}}
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
