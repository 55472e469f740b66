"""Pins of the oracle's SQP loop (Algorithm 1, Appendix D) and of its backward
pass (Algorithm 2, Appendix E):

* LQ: a second SQP step from a converged first step is a no-op;
* every accepted line-search step satisfies the Armijo condition of
  Appendix D or is the least-merit candidate;
* gradients of a loss through the converged FP64 solution map against central
  finite differences (hard active bounds, L1+L2 soft rows, slack weights,
  and a nonlinear model with the exact Lagrangian Hessian);
* unconstrained LQ: dL/dx_init equals the closed-loop Riccati sensitivity;
* inactive bounds get exactly zero gradient.
"""
import dataclasses

import numpy as np
import pytest

import workloads as w
from oracle import backward, models, sqp
from tests.test_oracle_admm import riccati_lq, tight


def test_lq_second_sqp_step_is_noop():
    p = w.double_integrator(N=10)
    inst = p.instance(0)
    o1 = tight(dataclasses.replace(p.opts, max_sqp=1))
    o2 = tight(dataclasses.replace(p.opts, max_sqp=2))
    s1 = sqp.solve(inst, o1)
    s2 = sqp.solve(inst, o2)
    assert np.max(np.abs(s1["z"] - s2["z"])) < 1e-9
    assert np.max(np.abs(s1["yf"] - s2["yf"])) < 1e-7


def test_linesearch_steps_satisfy_armijo():
    p = w.racing(B=1, N=12, track_length=150.0)
    inst = p.instance(0)
    s = sqp.solve(inst, p.opts, record=True)
    assert len(s["history"]) == p.opts.max_sqp
    for h in s["history"]:
        ls = h["ls"]
        a = h["alpha"]
        alphas = [2.0 ** (-k) for k in range(p.opts.n_ls)]
        k = alphas.index(a)
        armijo = ls["phis"][k] <= ls["phi0"] + p.opts.ls_eta * a * ls["D"]
        assert armijo or ls["phis"][k] == min(ls["phis"])
        assert ls["D"] < 0


def _loss_fd(inst, opts, dLdz, dLdxi, key, idx, h):
    vals = []
    for sgn in (1, -1):
        i2 = dict(inst)
        i2[key] = np.array(inst[key], dtype=float).copy()
        i2[key][idx] += sgn * h
        s = sqp.solve(i2, opts)
        vals.append(np.sum(dLdz * s["z"]) + np.sum(dLdxi * s["xi"]))
    return (vals[0] - vals[1]) / (2 * h)


def _check_fd(inst, opts, cases, h=1e-5, tol=2e-5, exact_hessian=False, seed=0):
    sol = sqp.solve(inst, opts)
    rng = np.random.default_rng(seed)
    dLdz = rng.normal(size=sol["z"].shape)
    dLdxi = rng.normal(size=sol["xi"].shape)
    gr, info = backward.backward(inst, sol, dLdz, dLdxi, eps_g=1e-7, exact_hessian=exact_hessian)
    for key, idx in cases:
        fd = _loss_fd(inst, opts, dLdz, dLdxi, key, idx, h)
        an = gr[key][idx]
        assert abs(fd - an) <= tol * max(1.0, abs(fd)), (key, idx, fd, an)
    return gr, info


def test_backward_fd_hard_active_bounds():
    p = w.tracking(B=1, nx=6, nu=3, N=8, seed=11)
    inst = p.instance(0)
    inst["x0"] = inst["x0"] * 6.0                          # drive the controls onto |u| <= 1
    opts = tight(p.opts, iters=60000, eps=1e-12)
    sol = sqp.solve(inst, opts)
    lower, upper, _ = backward.active_set(inst, sol["z"], sol["xi"], sol["yg"], 1e-7)
    act = np.argwhere(lower | upper)
    assert len(act) >= 3
    t0, i0 = act[0]
    cases = [("x0", (0,)), ("x0", (4,)), ("Qd", (3, 2)), ("Rd", (5, 1)), ("ref", (2, 4)),
             ("lin", (6, 7)), ("lo" if lower[t0, i0] else "hi", (t0, i0))]
    gr, info = _check_fd(inst, opts, cases)
    # inactive bounds: exactly zero
    inactive = ~(lower | upper)
    assert np.all(gr["lo"][inactive] == 0) and np.all(gr["hi"][inactive] == 0)


def test_backward_fd_soft_rows_and_gamma():
    p = w.double_integrator(N=6)
    inst = p.instance(0)
    inst["x0"] = np.array([0.5, -0.3, 3.0, -2.6])
    inst["gamma2"] = np.array([np.inf, np.inf, 4.0, 6.0])
    inst["gamma1"] = np.array([0.0, 0.0, 0.3, 0.2])
    inst["Wd"] = np.array([0.2, 0.1])                      # rate cost couples the stages
    opts = tight(p.opts, iters=80000, eps=1e-12)
    sol = sqp.solve(inst, opts)
    lower, upper, slack = backward.active_set(inst, sol["z"], sol["xi"], sol["yg"], 1e-7)
    assert slack.sum() >= 1
    ts, is_ = np.argwhere(slack)[0]
    cases = [("x0", (2,)), ("gamma2", (2,)), ("gamma1", (2,)), ("gamma2", (3,)),
             ("Wd", (0,)), ("Qd", (2, 1)), ("lo" if lower[ts, is_] else "hi", (ts, is_))]
    _check_fd(inst, opts, cases, tol=5e-5)


def test_backward_fd_nonlinear_exact_hessian():
    p = w.uneven(B=40, N_lo=5, N_hi=5, seed=21)
    i = int(np.flatnonzero(p.model == w.MODEL_QUAD)[0])
    inst = p.instance(i)
    inst["x0"] = np.array([0.3, -0.2, 0.25, 0.4, -0.3, 0.5])
    # full Gauss-Newton steps (n_ls = 1) converge linearly to the KKT point here
    opts = tight(dataclasses.replace(p.opts, max_sqp=30, n_ls=1, eps_c=1e-13), iters=20000, eps=1e-13)
    sol = sqp.solve(inst, opts)
    assert sol["stats"]["kkt"] < 1e-9
    cases = [("x0", (0,)), ("x0", (2,)), ("Qd", (3, 0)), ("Rd", (2, 1)), ("ref", (4, 6))]
    _check_fd(inst, opts, cases, h=1e-5, tol=1e-4, exact_hessian=True)


def test_backward_x0_matches_riccati_sensitivity():
    p = w.double_integrator(N=12)
    inst = p.instance(0)
    inst["lo"][:] = -np.inf
    inst["hi"][:] = np.inf
    N, nx = inst["N"], inst["nx"]
    A, B = models.di_matrices(inst["dyn"][0])
    opts = tight(p.opts)
    sol = sqp.solve(inst, opts)
    rng = np.random.default_rng(7)
    dLdz = rng.normal(size=sol["z"].shape)
    gr, _ = backward.backward(inst, sol, dLdz)
    Q = [np.diag(inst["Qd"][t]) for t in range(N)]
    R = [np.diag(inst["Rd"][t]) for t in range(N)]
    _, _, K = riccati_lq(A, B, Q, R, np.diag(inst["Qd"][N]), inst["x0"], N)
    # closed loop x_t = Phi_t x_init, u_t = -K_t Phi_t x_init, u_N = 0
    Phi = np.eye(nx)
    g = np.zeros(nx)
    for t in range(N + 1):
        g += Phi.T @ dLdz[t, :nx]
        if t < N:
            g += (-K[t] @ Phi).T @ dLdz[t, nx:]
            Phi = (A - B @ K[t]) @ Phi
    assert np.allclose(gr["x0"], g, atol=1e-7)


# ---------------------------------------------------------------------------
# The reduced adjoint QP of Appendix E (hard active rows as penalties gamma_xi)
# ---------------------------------------------------------------------------
def _hard_active_instance():
    p = w.tracking(B=1, nx=6, nu=3, N=8, seed=11)
    inst = p.instance(0)
    inst["x0"] = inst["x0"] * 6.0                          # controls on |u| <= 1
    sol = sqp.solve(inst, tight(p.opts, iters=60000, eps=1e-12))
    return inst, sol


def test_adjoint_qp_penalty_tends_to_the_exact_adjoint():
    """The bias of the penalised adjoint against the exact one (pinned by finite
    differences above) falls like 1 / gamma_xi."""
    inst, sol = _hard_active_instance()
    rng = np.random.default_rng(4)
    dLdz = rng.normal(size=sol["z"].shape)
    exact, info = backward.backward(inst, sol, dLdz, eps_g=1e-7)
    assert (info["lower"] | info["upper"]).sum() >= 3 and not info["slack"].any()
    errs = []
    for gam in (1e2, 1e4, 1e6):
        pen, _ = backward.backward(inst, sol, dLdz, eps_g=1e-7, penalty=gam)
        keys = ("x0", "Qd", "Rd", "ref", "lo", "hi")
        errs.append(max(np.linalg.norm(pen[k] - exact[k]) / max(np.linalg.norm(exact[k]), 1e-12) for k in keys))
    assert errs[0] > 1e-4
    assert 3e-3 < errs[1] / errs[0] < 3e-2 and 3e-3 < errs[2] / errs[1] < 3e-2


def test_adjoint_qp_penalty_equals_slack_rows_of_that_weight():
    """Eliminating a penalty row's multiplier (-1/gamma on its diagonal) is the
    same as giving the row an active slack of L2 weight gamma: the oracle's
    slack blocks (a separate assembly) reproduce the penalised adjoint."""
    inst, sol = _hard_active_instance()
    rng = np.random.default_rng(6)
    dLdz = rng.normal(size=sol["z"].shape)
    gam = 300.0
    pen, _ = backward.backward(inst, sol, dLdz, eps_g=1e-7, penalty=gam)
    lower, upper, _ = backward.active_set(inst, sol["z"], sol["xi"], sol["yg"], 1e-7)
    soft = dict(inst, gamma2=np.full_like(inst["gamma2"], gam), gamma1=np.zeros_like(inst["gamma1"]))
    orig = backward.active_set
    try:
        backward.active_set = lambda *a, **k: (lower, upper, lower | upper)
        via_slack, _ = backward.backward(soft, sol, dLdz, eps_g=1e-7)
    finally:
        backward.active_set = orig
    for k in ("x0", "Qd", "Rd", "ref", "lo", "hi", "lin", "Wd"):
        assert np.allclose(pen[k], via_slack[k], rtol=1e-9, atol=1e-12), k


def test_adjoint_qp_without_hard_active_rows_is_the_exact_adjoint():
    p = w.tracking(B=1, nx=6, nu=3, N=8, seed=11)
    inst = p.instance(0)
    inst["x0"] = inst["x0"] * 0.1                           # small x0: no bound active
    sol = sqp.solve(inst, tight(p.opts, iters=20000, eps=1e-12))
    dLdz = np.random.default_rng(8).normal(size=sol["z"].shape)
    a, info = backward.backward(inst, sol, dLdz, eps_g=1e-7)
    b, _ = backward.backward(inst, sol, dLdz, eps_g=1e-7, penalty=10.0)
    assert not (info["lower"] | info["upper"]).any()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
