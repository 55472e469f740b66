"""SQP outer loop of the paper (Algorithm 1), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  initial guess   the instance's z_init if it carries one (zero slacks and
                  multipliers), else x_0 = x_init, u_t = u_ref_t, each x_{t+1}
                  found from f_t(z_t, z_{t+1}) = 0 by `newton_steps` Newton
                  steps started from an explicit step (exact for explicit models);
  loop            convexify (oracle.qp) -> ADMM (oracle.admm, warm-started
                  from the current primal-dual point and the previous rho; on
                  the rescaled QP when the instance carries scales, Remark 4)
                  -> line search (Appendix D) -> convergence check (Eq. sqp_stop).

Line search (Appendix D): direction (dz, dxi) = (z*, xi*) - (z, xi); merit
  phi = l(z) + slack cost(xi) + mu V(z, xi),
  V   = ||f(z)||_1 + ||[g(z)+xi-hi]_+||_1 + ||[lo-g(z)-xi]_+||_1  (f includes x_0 - x_init),
  mu  = max( grad_l' d / (1/2 max(V, eps_c)),  ||y*||_inf + 1e-4 ),
  D   = grad_l' d - mu V;  candidates alpha = 2^-k, k = 0..n_ls-1, evaluated
  together; the largest with phi(alpha) <= phi(0) + eta alpha D is taken, else
  the finite candidate of least merit.  Multipliers move with the same step:
  y <- y + alpha (y* - y).
The floor ||y*||_inf + 1e-4 on mu (the exact-penalty condition) is this
implementation's reading where the printed ratio is not positive.
Parity: one SQP step of an LQ problem is pinned (a second step is a no-op,
the Armijo condition holds for the accepted step), a worked line search by
hand (tests/test_oracle_pins.py), and the converged nonlinear loop against an
independent NLP solver on small bicycle and quadrotor OCPs
(tests/test_oracle_nlp.py); the path at fixed counts is pinned only by the
algorithm itself.
"""
from __future__ import annotations

import math

import numpy as np

from . import admm as admm_mod
from . import models, qp as qp_mod


def rollout(inst, u=None, newton_steps=3):
    """Initial primal guess [N+1, n]: controls u (default u_ref), states by
    Newton's method on the dynamics residual of each stage."""
    nx, nu, N = inst["nx"], inst["nu"], inst["N"]
    z = np.zeros((N + 1, nx + nu))
    z[:, nx:] = inst["ref"][:, nx:] if u is None else u
    z[0, :nx] = inst["x0"]
    for t in range(N):
        xn = models.rollout_guess(inst, z[t, :nx], z[t, nx:])
        for _ in range(newton_steps):
            pair = np.stack([z[t], np.concatenate([xn, z[t + 1, nx:]])])
            f, _, Ap = models.dynamics(inst, pair)
            xn = xn - np.linalg.solve(Ap[0][:, :nx], f[0])
        z[t + 1, :nx] = xn
    return z


def constraint_violation(inst, z, xi):
    f, _, _ = models.dynamics(inst, z)
    g, _ = models.constraints(inst, z)
    gx = g + xi
    v = np.sum(np.abs(f)) + np.sum(np.abs(z[0, :inst["nx"]] - inst["x0"]))
    v += np.sum(np.maximum(gx - inst["hi"], 0.0)) + np.sum(np.maximum(inst["lo"] - gx, 0.0))
    return float(v)


def merit_parts(inst, z, xi):
    return models.cost(inst, z) + models.slack_cost(inst, xi), constraint_violation(inst, z, xi)


def directional_cost_derivative(inst, z, xi, dz, dxi):
    d = float(np.sum(models.cost_grad(inst, z) * dz))
    g2, g1 = inst["gamma2"], inst["gamma1"]
    soft = np.isfinite(g2)
    if np.any(soft):
        x, dx = xi[:, soft], dxi[:, soft]
        d += float(np.sum(g2[soft] * x * dx))
        d += float(np.sum(g1[soft] * np.where(x != 0.0, np.sign(x) * dx, np.abs(dx))))
    return d


def linesearch(inst, opts, z, xi, dz, dxi, ystar_inf):
    """Returns (alpha, info) per Appendix D."""
    l0, V0 = merit_parts(inst, z, xi)
    gd = directional_cost_derivative(inst, z, xi, dz, dxi)
    mu = max(gd / (0.5 * max(V0, opts.eps_c)), ystar_inf + 1e-4)
    phi0 = l0 + mu * V0
    D = gd - mu * V0
    best, best_phi = None, math.inf
    alphas = [2.0 ** (-k) for k in range(opts.n_ls)]
    phis = []
    for a in alphas:
        la, Va = merit_parts(inst, z + a * dz, xi + a * dxi)
        phis.append(la + mu * Va)
    chosen = None
    for a, ph in zip(alphas, phis):
        if math.isfinite(ph) and ph <= phi0 + opts.ls_eta * a * D:
            chosen = a
            break
    if chosen is None:
        for a, ph in zip(alphas, phis):
            if math.isfinite(ph) and ph < best_phi:
                best, best_phi = a, ph
        chosen = 0.0 if best is None else best
    return chosen, dict(mu=mu, phi0=phi0, D=D, phis=phis)


def kkt_residual(inst, z, xi, yf, yg):
    """max of the three quantities of Eq. (sqp_stop) at (z, xi, y): stationarity
    of the Lagrangian (incl. the slack rows), dynamics residual, bound violation."""
    nx = inst["nx"]
    f, Am, Ap = models.dynamics(inst, z)
    g, Gt = models.constraints(inst, z)
    grad = models.cost_grad(inst, z)
    grad[0, :nx] += yf[0]
    grad[:-1] += np.einsum("tij,ti->tj", Am, yf[1:])
    grad[1:] += np.einsum("tij,ti->tj", Ap, yf[1:])
    grad += np.einsum("tij,ti->tj", Gt, yg)
    stat = float(np.max(np.abs(grad)))
    rs = admm_mod.slack_dual_residual(xi.reshape(-1), yg.reshape(-1),
                                      np.tile(inst["gamma2"], z.shape[0]),
                                      np.tile(inst["gamma1"], z.shape[0]))
    if rs.size:
        stat = max(stat, float(np.max(np.abs(rs))))
    feas = float(max(np.max(np.abs(f)) if f.size else 0.0, np.max(np.abs(z[0, :nx] - inst["x0"]))))
    gx = g + xi
    viol = float(max(np.max(np.maximum(gx - inst["hi"], 0.0)), np.max(np.maximum(inst["lo"] - gx, 0.0))))
    return max(stat, feas, viol), dict(stationarity=stat, dynamics=feas, bounds=viol)


def solve(inst, opts, warm=None, replay=None, record=False, perturb_S=None):
    """Algorithm 1 on one instance.  warm: optional dict(z, xi, yf, yg, rho_bar).
    replay: optional dict(alpha=[...], rho=[{k: rho}, ...]) that forces the line
    search steps / rho schedule (decision replay); a missing "rho" key or a None
    entry leaves that decision to the algorithm; with record, a forced step
    still records the line-search quantities (merits, margins) along the
    replayed path.  perturb_S: passed to the ADMM (backward-error analysis
    only).  Returns dict(z, xi, yf, yg, rho_bar, stats, history)."""
    nx, ng, N = inst["nx"], inst["ng"], inst["N"]
    if warm is None and inst.get("z_init") is not None:
        # an instance that carries an initial primal guess starts from it (zero slacks / multipliers)
        warm = dict(z=inst["z_init"], xi=np.zeros((N + 1, ng)), yf=np.zeros((N + 1, nx)),
                    yg=np.zeros((N + 1, ng)))
    if warm is not None:
        z, xi = warm["z"].copy(), warm["xi"].copy()
        yf, yg = warm["yf"].copy(), warm["yg"].copy()
        rho_bar = warm.get("rho_bar", opts.rho0)
    else:
        z = rollout(inst, newton_steps=opts.newton_steps)
        xi = np.zeros((N + 1, ng))
        yf = np.zeros((N + 1, nx))
        yg = np.zeros((N + 1, ng))
        rho_bar = opts.rho0
    hist = []
    admm_iters = refactors = 0
    last = None
    for it in range(opts.max_sqp):
        qp = qp_mod.build_qp(inst, z)
        x0 = z.reshape(-1)
        zg0 = qp["G"] @ x0
        sched = None if replay is None or replay.get("rho") is None else replay["rho"][it]
        if inst.get("scale") is not None:   # normalised states and controls (Remark 4)
            res = admm_mod.admm_rescaled(qp, opts, inst["scale"], models.selector_rows(inst), x0, zg0,
                                         yf.reshape(-1), yg.reshape(-1), rho_bar,
                                         rho_schedule=sched, perturb_S=perturb_S)
        else:
            res = admm_mod.admm(qp, opts, x0, zg0, yf.reshape(-1), yg.reshape(-1), rho_bar,
                                rho_schedule=sched, perturb_S=perturb_S)
        rho_bar = res["rho_bar"]
        admm_iters += res["iters"]
        refactors += res["refactors"]
        zs = res["x"].reshape(N + 1, -1)
        xis = res["xi"].reshape(N + 1, ng)
        yfs = res["yf"].reshape(N + 1, nx)
        ygs = res["yg"].reshape(N + 1, ng)
        ystar_inf = float(max(np.max(np.abs(yfs)), np.max(np.abs(ygs)) if ygs.size else 0.0))
        forced = None
        if replay is not None and replay.get("alpha") is not None and it < len(replay["alpha"]):
            forced = replay["alpha"][it]
        if forced is not None:
            a = forced
            info = linesearch(inst, opts, z, xi, zs - z, xis - xi, ystar_inf)[1] if record else {}
        else:
            a, info = linesearch(inst, opts, z, xi, zs - z, xis - xi, ystar_inf)
        z = z + a * (zs - z)
        xi = xi + a * (xis - xi)
        yf = yf + a * (yfs - yf)
        yg = yg + a * (ygs - yg)
        last = res
        kkt, parts = kkt_residual(inst, z, xi, yf, yg)
        hist.append(dict(alpha=a, kkt=kkt, r_prim=res["r_prim"], r_dual=res["r_dual"],
                         rho_bar=rho_bar, rho_events=res["rho_events"], admm_iters=res["iters"],
                         **({"ls": info} if record else {})))
        if opts.early_exit and kkt <= opts.eps_c:
            break
    kkt, parts = kkt_residual(inst, z, xi, yf, yg)
    stats = dict(sqp_iters=len(hist), admm_iters=admm_iters, r_prim=last["r_prim"],
                 r_dual=last["r_dual"], prim_norm=last["prim_norm"], dual_norm=last["dual_norm"],
                 rho_bar=rho_bar, refactors=refactors, kkt=kkt, **parts)
    return dict(z=z, xi=xi, yf=yf, yg=yg, rho_bar=rho_bar, stats=stats, history=hist)
