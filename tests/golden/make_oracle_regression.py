"""Writes oracle_regression.json: outputs of the FP64 oracle on a small
seeded case, kept as a regression guard for the oracle itself.

The paper prints no worked example, so these are not paper values: they are
the oracle's own results (this script calls only oracle/ and the seeded
input generator), stored so that an accidental change of the oracle's
arithmetic shows up as a failing test. A deliberate change regenerates the
file and names the passage that justifies it.

  python tests/golden/make_oracle_regression.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2108_07031_gb300 import cloud as Cl  # noqa: E402


def compute():
    c = Cl.naca0012_cloud(24, 8)
    oc = O.OracleCloud.from_cloud(c)
    W = Cl.perturbed_state(c, 0.63, 2.0)
    R, bad = O.residual_of_state(oc, W, inner=2)
    W0 = np.tile(O.freestream(0.63, 2.0), (c.n, 1))
    W50, res, st = O.iterate(oc, W0, 50)
    cl, cd = O.forces(oc, W50, c.wall_loop, 0.63, 2.0)
    return {
        "case": "24 x 8 NACA 0012 cloud (cloud.naca0012_cloud(24, 8)), M 0.63, alpha 2 deg",
        "residual_of_perturbed_state": R.tolist(),
        "bad_stencils": int(bad),
        "iterate_50_from_freestream": {"state": W50.tolist(), "residue": list(map(float, res)),
                                        "status": int(st), "cl": float(cl), "cd": float(cd)},
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(compute(), f)
    print("wrote", os.path.join(HERE, "oracle_regression.json"))
