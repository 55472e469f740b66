"""Pin of the oracle's nonlinear SQP loop (Algorithm 1: linearisation, QP in
absolute coordinates, ADMM, merit line search, multiplier steps) as a whole:
run to convergence on small nonlinear OCPs with active hard bounds, it must
reach the minimiser that an independent NLP solver (SciPy's SLSQP on the same
cost, dynamics and bounds, written from the model functions that the
finite-difference pins of test_oracle_models.py fix) finds, and its KKT
residual of Eq. (sqp_stop) must vanish.  A mistake in the QP's coordinates,
the step or the multiplier update moves the fixed point or stops convergence.
"""
import dataclasses

import numpy as np
import pytest
from scipy.optimize import minimize

import workloads as w
from oracle import models, sqp


def _nlp_minimiser(inst, z_start):
    N, nx, n = inst["N"], inst["nx"], inst["nx"] + inst["nu"]
    unpack = lambda v: v.reshape(N + 1, n)

    def eq(v):
        z = unpack(v)
        f, _, _ = models.dynamics(inst, z)
        return np.concatenate([z[0, :nx] - inst["x0"], f.reshape(-1)])

    def eq_jac(v):   # [I 0] on x_0, then df_t / d(z_t, z_t+1) per stage
        _, Am, Ap = models.dynamics(inst, unpack(v))
        J = np.zeros((nx * (N + 1), n * (N + 1)))
        J[:nx, :nx] = np.eye(nx)
        for t in range(N):
            J[nx * (t + 1):nx * (t + 2), n * t:n * (t + 1)] = Am[t]
            J[nx * (t + 1):nx * (t + 2), n * (t + 1):n * (t + 2)] = Ap[t]
        return J

    lo, hi = inst["lo"], inst["hi"]
    mh, ml = np.isfinite(hi), np.isfinite(lo)

    def ineq(v):
        g, _ = models.constraints(inst, unpack(v))
        return np.concatenate([(hi - g)[mh], (g - lo)[ml]])

    def ineq_jac(v):
        _, G = models.constraints(inst, unpack(v))
        ng = G.shape[1]
        J = np.zeros(((N + 1) * ng, (N + 1) * n))
        for t in range(N + 1):
            J[ng * t:ng * (t + 1), n * t:n * (t + 1)] = G[t]
        return np.vstack([-J[mh.reshape(-1)], J[ml.reshape(-1)]])

    r = minimize(lambda v: models.cost(inst, unpack(v)), z_start.reshape(-1),
                 jac=lambda v: models.cost_grad(inst, unpack(v)).reshape(-1), method="SLSQP",
                 constraints=[{"type": "eq", "fun": eq, "jac": eq_jac},
                              {"type": "ineq", "fun": ineq, "jac": ineq_jac}],
                 options=dict(maxiter=3000, ftol=1e-15))
    assert r.success, r.message
    return unpack(r.x)


def _tight(opts, sqp_iters):
    return dataclasses.replace(opts, max_sqp=sqp_iters, max_admm=40000, early_exit=1, eps_abs=1e-11,
                               eps_rel=1e-11, eps_c=1e-9, check_every=25)


def _active(inst, z):
    g, _ = models.constraints(inst, z)
    return int(np.sum(np.isclose(g, inst["hi"], atol=1e-6) | np.isclose(g, inst["lo"], atol=1e-6)))


def test_sqp_reaches_the_nlp_minimiser_bicycle():
    """Implicit-midpoint bicycle on a short track, every row hard, the speed bound
    active below the initial speed."""
    pb = w.racing(B=1, N=6, track_length=60.0)
    inst = pb.instance(0)
    inst["gamma2"] = np.full_like(inst["gamma2"], np.inf)
    inst["gamma1"] = np.zeros_like(inst["gamma1"])
    inst["hi"][1:, 2] = inst["z_init"][0, 3] - 0.1
    o = sqp.solve(inst, _tight(pb.opts, 80))
    ref = _nlp_minimiser(inst, inst["z_init"])
    assert o["stats"]["kkt"] < 1e-9
    assert _active(inst, o["z"]) >= 1
    assert np.max(np.abs(o["z"] - ref)) / max(1.0, np.max(np.abs(ref))) < 1e-6


def test_sqp_reaches_the_nlp_minimiser_quadrotor():
    """RK4 planar quadrotor pushed off hover, with a thrust bound active."""
    pb = w.uneven(B=40, N_lo=6, N_hi=6, seed=21)
    inst = pb.instance(int(np.flatnonzero(pb.model == w.MODEL_QUAD)[0]))
    inst["x0"] = inst["x0"] + np.array([0.3, -0.2, 0.2, 0.5, -0.3, 0.1])
    o = sqp.solve(inst, _tight(pb.opts, 60))
    ref = _nlp_minimiser(inst, sqp.rollout(inst))
    assert o["stats"]["kkt"] < 1e-6
    assert _active(inst, o["z"]) >= 1
    assert np.max(np.abs(o["z"] - ref)) / max(1.0, np.max(np.abs(ref))) < 1e-5


def test_rescaled_sqp_reaches_the_same_minimiser():
    """With the ADMM on the rescaled QP (normalised states and controls), the
    converged SQP point is still the NLP minimiser: the rescaling changes the
    inner iteration, not the problem."""
    pb = w.racing(B=1, N=6, track_length=60.0)
    inst = pb.instance(0)
    inst["gamma2"] = np.full_like(inst["gamma2"], np.inf)
    inst["gamma1"] = np.zeros_like(inst["gamma1"])
    inst["hi"][1:, 2] = inst["z_init"][0, 3] - 0.1
    pb.scale = w.magnitude_scales(pb)
    inst["scale"] = pb.scale[0]
    o = sqp.solve(inst, _tight(pb.opts, 80))
    ref = _nlp_minimiser(inst, inst["z_init"])
    assert o["stats"]["kkt"] < 1e-7     # the inner tolerance now acts in scaled units
    assert np.max(np.abs(o["z"] - ref)) / max(1.0, np.max(np.abs(ref))) < 1e-6


@pytest.mark.parametrize("integrator", ["trapezoidal", "newton_map"])
def test_sqp_reaches_the_nlp_minimiser_other_time_discretisations(integrator):
    """The bicycle under the trapezoidal constraint (A^+ with a control block) and
    under the explicit map that 3 Newton steps on the midpoint rule define (IFT
    Jacobians)."""
    pb = w.racing(B=1, N=6, track_length=60.0, integrator=integrator)
    inst = pb.instance(0)
    inst["gamma2"] = np.full_like(inst["gamma2"], np.inf)
    inst["gamma1"] = np.zeros_like(inst["gamma1"])
    inst["hi"][1:, 2] = inst["z_init"][0, 3] - 0.1
    o = sqp.solve(inst, _tight(pb.opts, 80))
    ref = _nlp_minimiser(inst, inst["z_init"])
    assert o["stats"]["kkt"] < 1e-6
    assert _active(inst, o["z"]) >= 1
    assert np.max(np.abs(o["z"] - ref)) / max(1.0, np.max(np.abs(ref))) < 1e-6


def test_sqp_reaches_the_nlp_minimiser_srb_humanoid():
    """Single-rigid-body humanoid (RK4, n = 18) with the vertical foot forces capped
    below the weight, so that the cap is active on every stage."""
    pb = w.humanoid(B=1, N=5)
    inst = pb.instance(0)
    inst["hi"][:, 2] = 150.0
    inst["hi"][:, 5] = 150.0
    o = sqp.solve(inst, _tight(pb.opts, 60))
    z0 = inst["z_init"] if inst.get("z_init") is not None else sqp.rollout(inst)
    ref = _nlp_minimiser(inst, z0)
    assert o["stats"]["kkt"] < 1e-6
    assert _active(inst, o["z"]) >= 6
    assert np.max(np.abs(o["z"] - ref)) / max(1.0, np.max(np.abs(ref))) < 1e-6


def _nlp_minimiser_with_slacks(inst, z_start):
    """The same NLP with the L1 + L2 slack of every soft row, the slack split as
    xi = p - m with p, m >= 0 so that gamma1 |xi| = gamma1 (p + m) is smooth:
    min l(z) + sum gamma2/2 xi^2 + gamma1 (p + m)  s.t. dynamics, lo <= g + xi <= hi."""
    N, nx, n = inst["N"], inst["nx"], inst["nx"] + inst["nu"]
    ks = np.flatnonzero(np.isfinite(inst["gamma2"]))
    ns = len(ks)
    nz, nsl = n * (N + 1), ns * (N + 1)
    g2, g1 = inst["gamma2"][ks], inst["gamma1"][ks]
    lo, hi = inst["lo"], inst["hi"]
    mh, ml = np.isfinite(hi), np.isfinite(lo)

    def split(v):
        return v[:nz].reshape(N + 1, n), v[nz:nz + nsl].reshape(N + 1, ns), v[nz + nsl:].reshape(N + 1, ns)

    def obj(v):
        z, p, m = split(v)
        xi = p - m
        return models.cost(inst, z) + np.sum(0.5 * g2 * xi ** 2 + g1 * (p + m))

    def obj_grad(v):
        z, p, m = split(v)
        xi = p - m
        return np.concatenate([models.cost_grad(inst, z).reshape(-1), (g2 * xi + g1).reshape(-1),
                               (-g2 * xi + g1).reshape(-1)])

    def eq(v):
        z = split(v)[0]
        f, _, _ = models.dynamics(inst, z)
        return np.concatenate([z[0, :nx] - inst["x0"], f.reshape(-1)])

    def ineq(v):
        z, p, m = split(v)
        g, _ = models.constraints(inst, z)
        g = g.copy()
        g[:, ks] += p - m
        return np.concatenate([(hi - g)[mh], (g - lo)[ml]])

    v0 = np.concatenate([z_start.reshape(-1), np.zeros(2 * nsl)])
    r = minimize(obj, v0, jac=obj_grad, method="SLSQP", bounds=[(None, None)] * nz + [(0.0, None)] * (2 * nsl),
                 constraints=[{"type": "eq", "fun": eq}, {"type": "ineq", "fun": ineq}],
                 options=dict(maxiter=5000, ftol=1e-15))
    z, p, m = split(r.x)
    xi = np.zeros((N + 1, inst["ng"]))
    xi[:, ks] = p - m
    return z, xi


def test_sqp_reaches_the_nlp_minimiser_with_l1_l2_slacks():
    """The racing track row kept soft (gamma2 = 100, gamma1 = 10) and narrowed so
    that its slack is used: the SQP's converged point and slacks equal the
    minimiser of the NLP with explicit slack variables."""
    pb = w.racing(B=1, N=4, track_length=60.0)
    inst = pb.instance(0)
    inst["lo"][1:, 4], inst["hi"][1:, 4] = -0.05, 0.05   # state rows bound t >= 1 (x_0 is fixed)
    inst["x0"] = inst["x0"] + np.array([0.0, 0.4, 0.05, 0.0, 0.0, 0.0])
    o = sqp.solve(inst, _tight(pb.opts, 80))
    z, xi = _nlp_minimiser_with_slacks(inst, inst["z_init"])
    assert o["stats"]["kkt"] < 1e-6
    assert np.max(np.abs(o["xi"])) > 1e-2
    assert np.max(np.abs(o["z"] - z)) / max(1.0, np.max(np.abs(z))) < 1e-5
    assert np.max(np.abs(o["xi"] - xi)) < 1e-5 * max(1.0, np.max(np.abs(xi)))
