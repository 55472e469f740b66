"""Pins of the oracle's rescaled ADMM (normalised states and controls, Remark 4)
against results fixed independently of the rescaling code:

* the rescaled ADMM converges to the brute-force solution of a tiny QP (hard
  rows, and L2-soft rows whose penalty the rescaling must carry over), with
  scales that differ per component;
* at convergence the primal point, the slacks and both multipliers equal the
  unscaled ADMM's on a racing QP (the change of variables leaves the KKT point
  where it is; a wrong unscaling of any of them fails);
* unit scales change nothing, bit for bit;
* a uniform scale d on a problem whose rows all bound single variables is, at
  a fixed iteration count (rho rule included), the plain ADMM on the cost
  multiplied by d^2 (ADMM is unchanged when the objective, rho and sigma are
  scaled together, and the change of variables divides rho and sigma by d^2);
  the multipliers come back divided by d^2.  This fixes the power of d on every
  piece of data (P, q, c, bounds, slack weights, multipliers).
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as w
from oracle import admm, models, qp as qpm, sqp

from test_oracle_admm import brute_force_qp, tight


def _rescaled(q, opts, d, sel, z0, rho=0.1):
    return admm.admm_rescaled(q, opts, np.asarray(d, float), np.asarray(sel), z0.reshape(-1),
                              q["G"] @ z0.reshape(-1), np.zeros(q["C"].shape[0]), np.zeros(q["G"].shape[0]), rho)


def test_pow2_floor():
    s = np.array([1.0, 0.75, 100.0, 0.5, 3.999, 4.0, 1e-3])
    assert np.array_equal(admm.pow2_floor(s), [1.0, 0.5, 64.0, 0.5, 2.0, 4.0, 2.0 ** -10])


D_MIXED = [4.0, 0.5, 2.0, 8.0, 0.25, 16.0]   # x, y, vx, vy, ux, uy of the double integrator


def test_rescaled_hard_qp_matches_brute_force():
    p = w.double_integrator(N=2)
    inst = p.instance(0)
    inst["x0"] = np.array([0.5, -0.3, 1.9, -1.8])
    inst["hi"][:, 0:2] = 0.4
    inst["lo"][:, 0:2] = -0.4
    z0 = sqp.rollout(inst)
    q = qpm.build_qp(inst, z0)
    zb, _ = brute_force_qp(q)
    r = _rescaled(q, tight(p.opts), D_MIXED, models.selector_rows(inst), z0)
    assert np.max(np.abs(r["x"] - zb)) < 1e-7


def test_rescaled_soft_qp_matches_brute_force():
    p = w.double_integrator(N=2)
    inst = p.instance(0)
    inst["x0"] = np.array([0.5, -0.3, 2.5, -2.4])
    inst["gamma2"] = np.array([np.inf, np.inf, 3.0, 5.0])
    inst["gamma1"] = np.zeros(4)
    z0 = sqp.rollout(inst)
    q = qpm.build_qp(inst, z0)
    soft_rows = [i for i in range(q["G"].shape[0]) if np.isfinite(q["gamma2"][i])
                 and (np.isfinite(q["lo"][i]) or np.isfinite(q["hi"][i]))]
    zb, xib = brute_force_qp(q, soft_rows)
    r = _rescaled(q, tight(p.opts), D_MIXED, models.selector_rows(inst), z0)
    assert np.max(np.abs(r["x"] - zb)) < 1e-7
    assert np.max(np.abs(r["xi"][soft_rows] - xib)) < 1e-7
    assert np.max(np.abs(xib)) > 1e-3
    g2 = q["gamma2"]
    m = np.isfinite(g2)
    assert np.max(np.abs(g2[m] * r["xi"][m] + r["yg"][m])) < 1e-9   # gamma xi + y = 0 in physical units


def test_rescaled_racing_qp_has_the_unscaled_kkt_point():
    p = w.racing(B=1, N=8, track_length=100.0)
    inst = p.instance(0)
    z0 = inst["z_init"]
    inst["hi"][1:, 2] = z0[0, 3] - 0.1               # speed bound below the guess's speed (reachable)
    inst["lo"][:, 4], inst["hi"][:, 4] = -0.05, 0.05  # narrow soft track row
    inst["x0"] = inst["x0"] + np.array([0.0, 0.3, 0.05, 0.0, 0.0, 0.0])
    q = qpm.build_qp(inst, z0)
    opts = tight(p.opts, iters=60000, eps=1e-11)
    x0, zg0 = z0.reshape(-1), q["G"] @ z0.reshape(-1)
    yf0, yg0 = np.zeros(q["C"].shape[0]), np.zeros(q["G"].shape[0])
    ref = admm.admm(q, opts, x0, zg0, yf0, yg0, 0.1)
    d = w.magnitude_scales(p)[0]
    r = admm.admm_rescaled(q, opts, d, models.selector_rows(inst), x0, zg0, yf0, yg0, 0.1)
    assert ref["converged"] and r["converged"]
    assert np.any(admm.pow2_floor(d) != 1.0)
    for k in ("x", "xi", "yf", "yg"):
        scale = max(1.0, np.max(np.abs(ref[k])))
        assert np.max(np.abs(r[k] - ref[k])) / scale < 1e-6, k
    assert np.max(np.abs(ref["yg"])) > 1e-2 and np.max(np.abs(ref["xi"])) > 1e-4   # bounds and slacks in use


def test_unit_scales_change_nothing():
    p = w.racing(B=1, N=8, track_length=100.0)
    inst = p.instance(0)
    z0 = inst["z_init"]
    q = qpm.build_qp(inst, z0)
    opts = dataclasses.replace(p.opts, max_admm=60)
    a = admm.admm(q, opts, z0.reshape(-1), q["G"] @ z0.reshape(-1), np.zeros(q["C"].shape[0]),
                  np.zeros(q["G"].shape[0]), 0.1)
    b = _rescaled(q, opts, np.ones(8), models.selector_rows(inst), z0)
    for k in ("x", "zg", "xi", "yf", "yg", "rho_bar", "r_prim", "r_dual"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("dscale", [4.0, 0.125])
def test_uniform_scale_is_a_scaled_cost_at_a_fixed_count(dscale):
    p = w.double_integrator(N=6)
    inst = p.instance(0)
    inst["x0"] = np.array([0.5, -0.3, 2.5, -2.4])
    inst["gamma2"] = np.array([np.inf, np.inf, 3.0, 5.0])    # soft velocity rows (L1 + L2)
    inst["gamma1"] = np.array([0.0, 0.0, 0.5, 0.2])
    z0 = sqp.rollout(inst)
    q = qpm.build_qp(inst, z0)
    opts = dataclasses.replace(p.opts, max_admm=90, k_rho_iter=25)
    rng = np.random.default_rng(5)
    x0, zg0 = z0.reshape(-1), q["G"] @ z0.reshape(-1)
    yf0, yg0 = rng.normal(size=q["C"].shape[0]), rng.normal(size=q["G"].shape[0])
    r = admm.admm_rescaled(q, opts, np.full(6, dscale), models.selector_rows(inst), x0, zg0, yf0, yg0, 0.1)
    d2 = dscale * dscale
    qc = dict(q, P=(d2 * q["P"]).tocsr(), q=d2 * q["q"], gamma2=d2 * q["gamma2"], gamma1=d2 * q["gamma1"])
    c = admm.admm(qc, opts, x0, zg0, d2 * yf0, d2 * yg0, 0.1)
    assert c["rho_events"] and r["rho_events"] == c["rho_events"]
    for k in ("x", "zg", "xi"):
        assert np.allclose(r[k], c[k], rtol=1e-9, atol=1e-12), k
    for k in ("yf", "yg"):
        assert np.allclose(r[k], c[k] / d2, rtol=1e-9, atol=1e-12), k
    assert np.max(np.abs(r["xi"])) > 1e-3


def test_selector_rows_are_the_unit_rows_of_g():
    """The rows the rescaling divides by one variable's scale are exactly the
    rows of G_t with a single unit entry in that column, for every model."""
    for p in (w.double_integrator(N=3), w.racing(B=1, N=4, track_length=60.0), w.uneven(B=8, seed=3)):
        for i in range(p.B):
            inst = p.instance(i)
            z = inst["z_init"] if inst.get("z_init") is not None else sqp.rollout(inst)
            _, G = models.constraints(inst, z)
            sel = models.selector_rows(inst)
            for r, j in enumerate(sel):
                if j >= 0:
                    e = np.zeros(G.shape[2]); e[j] = 1.0
                    assert np.all(G[:, r, :] == e)
                else:
                    assert np.any(np.count_nonzero(G[:, r, :], axis=1) > 1)


def test_rescaled_blocks_keep_their_unit_structure():
    """The reading divides each dynamics row by the scale of the state it
    defines and each box row by its variable's scale, so that the scaled
    blocks keep the structure the stage-wise solvers rely on: the initial
    condition [I 0], the explicit model's A^+ = [-I 0], the implicit midpoint
    rule's A^+_x = A^-_x - 2 I, and unit selector rows of G."""
    d = np.array([4.0, 0.5, 2.0, 8.0, 0.25, 16.0, 2.0, 32.0])
    for p in (w.double_integrator(N=3), w.racing(B=1, N=4, track_length=60.0)):
        inst = p.instance(0)
        nx, n, N = inst["nx"], inst["nx"] + inst["nu"], inst["N"]
        z = inst["z_init"] if inst.get("z_init") is not None else sqp.rollout(inst)
        q = qpm.build_qp(inst, z)
        sq, Dv, Ef, Eg = admm.rescale_qp(q, d[:n], models.selector_rows(inst))
        C = sq["C"].toarray()
        assert np.array_equal(C[:nx, :n], np.hstack([np.eye(nx), np.zeros((nx, n - nx))]))
        for t in range(N):
            Am = C[(t + 1) * nx:(t + 2) * nx, t * n:(t + 1) * n]
            Ap = C[(t + 1) * nx:(t + 2) * nx, (t + 1) * n:(t + 2) * n]
            assert np.all(Ap[:, nx:] == 0)
            if inst["model"] == w.MODEL_DI:
                assert np.array_equal(Ap[:, :nx], -np.eye(nx))
            else:
                assert np.allclose(Ap[:, :nx], Am[:, :nx] - 2.0 * np.eye(nx), rtol=0, atol=1e-13)
        G = sq["G"].toarray()
        ng = inst["ng"]
        for t in range(N + 1):
            for r, j in enumerate(models.selector_rows(inst)):
                if j >= 0:
                    e = np.zeros(n); e[j] = 1.0
                    assert np.array_equal(G[t * ng + r, t * n:(t + 1) * n], e)


def test_magnitude_scales_of_the_workloads():
    """The input helper: per component the largest |value| in the initial guess
    or of a finite bound on a row that bounds the component alone, floored at 1."""
    pb = w.racing(B=2, N=10, track_length=80.0)
    m = w.magnitude_scales(pb)
    for i in range(pb.B):
        T = int(pb.N[i]) + 1
        guess = np.max(np.abs(pb.z_init[i, :T, :8]), axis=0)
        assert m[i, 3] == max(1.0, guess[3], 30.0)          # speed: bound 30 m/s
        assert m[i, 6] == max(1.0, guess[6], 4.0)           # acceleration: |a| <= 4
        assert m[i, 0] == max(1.0, guess[0])                # x position: no bound row
        assert np.all(m[i] >= 1.0)
