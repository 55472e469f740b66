"""Writes tests/golden/oracle_regression.json: FP64 oracle solutions of small
seeded instances, used as regression fixtures (the oracle must keep
reproducing them) and as stored expected values for the GPU parity tests.
Calls only the oracle and the seeded generators.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), "..", ".."))
sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402
from oracle import sqp  # noqa: E402

CASES = {
    # the double-integrator workload exactly as configured (1 SQP x 200 ADMM)
    "double_integrator_B1_N20": lambda: w.double_integrator(B=1, N=20),
    # a short racing instance, 2 SQP x 20 ADMM, from the centreline guess
    "racing_B1_N10": lambda: w.racing(B=1, N=10, max_sqp=2, max_admm=20),
}


def compute():
    out = {}
    for name, make in CASES.items():
        pb = make()
        o = sqp.solve(pb.instance(0), pb.opts)
        st = o["stats"]
        out[name] = {"z": o["z"].tolist(), "xi": o["xi"].tolist(), "yf": o["yf"].tolist(), "yg": o["yg"].tolist(),
                     "stats": {k: float(st[k]) for k in ("sqp_iters", "admm_iters", "r_prim", "r_dual",
                                                          "prim_norm", "dual_norm", "rho_bar", "kkt")}}
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(__file__), "oracle_regression.json")
    with open(path, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", path)
