"""Stored oracle solutions (tests/golden/oracle_regression.json, written by
tests/golden/make_golden.py from the oracle only): the oracle keeps
reproducing them, and the GPU path matches them at the stored sizes."""
import json
import os

import numpy as np
import pytest

import workloads as w

HERE = os.path.dirname(__file__)
GOLD = json.load(open(os.path.join(HERE, "golden", "oracle_regression.json")))


def test_oracle_reproduces_the_stored_solutions():
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden
    now = make_golden.compute()
    for name, ref in GOLD.items():
        for k in ("z", "xi", "yf", "yg"):
            np.testing.assert_allclose(np.array(now[name][k]), np.array(ref[k]), rtol=1e-9, atol=1e-11, err_msg=name + k)
        assert now[name]["stats"]["admm_iters"] == ref["stats"]["admm_iters"]


@pytest.mark.gpu
def test_gpu_matches_the_stored_double_integrator_solution():
    import torch
    from paper_2606_24039_gb300 import Solver, build
    build.build()
    pb = w.double_integrator(B=1, N=20)
    ref = GOLD["double_integrator_B1_N20"]
    for solver in (1, 2, 4):
        s = Solver.from_batch(pb, device="cuda", solver=solver)
        sol = s.tmpc_solve(s.x0)
        torch.cuda.synchronize()
        z = sol["z"][0].cpu().numpy()
        zr = np.array(ref["z"])
        assert np.max(np.abs(z - zr)) / max(1.0, np.max(np.abs(zr))) <= 1e-4, solver
        assert abs(float(sol["stats"][0, 2]) - ref["stats"]["r_prim"]) <= 1e-5 * max(1.0, ref["stats"]["prim_norm"])
