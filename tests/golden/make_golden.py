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


def compute(name):
    cfg = CASES[name]()
    J, gth, info = S.loss_and_grad(cfg, tol=1e-13)
    return {"loss": J, "dJ_dtheta": [float(x) for x in gth], "steps": len(info["tapes"])}


def main():
    out = {"generator": "tests/golden/make_golden.py", "tol": 1e-13,
           "cases": {k: compute(k) for k in CASES}}
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
