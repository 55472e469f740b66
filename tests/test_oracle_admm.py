"""Pins of the oracle's QP assembly and ADMM (Algorithm 3) against results the
mathematics fixes independently of the oracle:

* the block formulas of S (Appendix C) equal P + sigma I + A' rho A of the
  assembled matrices;
* the QP of a quadratic cost is the cost itself (q_abs, P against a direct
  cost evaluation), the linearised dynamics of a linear model are exact;
* unconstrained LQ: ADMM converges to the discrete Riccati solution;
* tiny constrained QPs: ADMM converges to the solution found by brute-force
  enumeration of active sets of the dense KKT system (hard and L2-soft rows);
* the (smoothed) projection equals the printed formula Eq. (proj:tilde) when
  gamma1 = 0, minimises its objective for gamma1 > 0, and tends to the hard
  projection as gamma2 grows;
* invariants after the last update: gamma xi + y = 0 on soft rows, and the
  primal/dual residuals vanish at convergence.
"""
import dataclasses
import itertools

import numpy as np
import pytest

import workloads as w
from oracle import admm, models, qp as qpm, sqp


def tight(opts, iters=20000, eps=1e-12):
    return dataclasses.replace(opts, max_admm=iters, early_exit=1, eps_abs=eps, eps_rel=eps,
                               check_every=25)


def test_schur_block_formulas_match_assembled_S():
    for p in [w.racing(B=1, N=6, track_length=100.0), w.tracking(B=1, nx=5, nu=3, N=5)]:
        inst = p.instance(0)
        z = sqp.rollout(inst)
        q = qpm.build_qp(inst, z)
        S = admm.form_S(q, 1e-6, 37.0, 0.7).toarray()
        Th, Ph = qpm.schur_blocks(q, 1e-6, 37.0, 0.7)
        n, N = q["n"], q["N"]
        for t in range(N + 1):
            assert np.allclose(S[t * n:(t + 1) * n, t * n:(t + 1) * n], Th[t], atol=1e-10)
        for t in range(N):
            assert np.allclose(S[(t + 1) * n:(t + 2) * n, t * n:(t + 1) * n], Ph[t], atol=1e-10)
        # nothing outside the block tridiagonal band
        for t in range(N + 1):
            for s in range(N + 1):
                if abs(t - s) > 1:
                    assert np.all(S[t * n:(t + 1) * n, s * n:(s + 1) * n] == 0)


def test_qp_model_of_quadratic_cost_is_exact():
    p = w.racing(B=1, N=6, track_length=100.0)
    inst = p.instance(0)
    rng = np.random.default_rng(2)
    z0 = sqp.rollout(inst)
    q1 = qpm.build_qp(inst, z0)
    q2 = qpm.build_qp(inst, z0 + rng.normal(size=z0.shape))
    # the absolute-coordinate linear term does not depend on the iterate
    assert np.allclose(q1["q"], q2["q"], atol=1e-10)
    assert np.allclose((q1["P"] - q2["P"]).toarray(), 0)
    # 1/2 z'Pz + q'z differs from the cost by a constant
    diffs = []
    for _ in range(4):
        z = rng.normal(size=z0.shape)
        zf = z.reshape(-1)
        diffs.append(models.cost(inst, z) - (0.5 * zf @ (q1["P"] @ zf) + q1["q"] @ zf))
    assert np.ptp(diffs) < 1e-8


def test_linear_model_constraints_are_exact():
    p = w.tracking(B=1, nx=5, nu=3, N=5)
    inst = p.instance(0)
    rng = np.random.default_rng(3)
    q = qpm.build_qp(inst, rng.normal(size=(6, 8)))
    z = rng.normal(size=(6, 8))
    f, _, _ = models.dynamics(inst, z)
    res = q["C"] @ z.reshape(-1) - q["c"]
    assert np.allclose(res[:5], z[0, :5] - inst["x0"])
    assert np.allclose(res[5:], f.reshape(-1))


def riccati_lq(A, B, Q, R, Qf, x0, N):
    """Textbook finite-horizon discrete Riccati recursion for
    min sum_t 1/2 x'Q_t x + 1/2 u'R_t u + 1/2 x_N' Qf x_N, x+ = A x + B u."""
    P = Qf
    K = [None] * N
    for t in range(N - 1, -1, -1):
        K[t] = np.linalg.solve(R[t] + B.T @ P @ B, B.T @ P @ A)
        P = Q[t] + A.T @ P @ (A - B @ K[t])
    xs, us = [x0], []
    for t in range(N):
        us.append(-K[t] @ xs[-1])
        xs.append(A @ xs[-1] + B @ us[-1])
    return np.array(xs), np.array(us), K


@pytest.mark.parametrize("which", ["double_integrator", "linear"])
def test_unconstrained_lq_matches_riccati(which):
    if which == "double_integrator":
        p = w.double_integrator(N=20)
        inst = p.instance(0)
        A, B = models.di_matrices(inst["dyn"][0])
    else:
        p = w.tracking(B=1, nx=6, nu=3, N=15)
        inst = p.instance(0)
        inst["ref"][:] = 0.0
        A, B, _ = models.linear_matrices(inst)
    inst["lo"][:] = -np.inf
    inst["hi"][:] = np.inf
    N = inst["N"]
    nx = inst["nx"]
    sol = sqp.solve(inst, tight(p.opts))
    Q = [np.diag(inst["Qd"][t]) for t in range(N)]
    R = [np.diag(inst["Rd"][t]) for t in range(N)]
    xs, us, _ = riccati_lq(A, B, Q, R, np.diag(inst["Qd"][N]), inst["x0"], N)
    assert np.allclose(sol["z"][:, :nx], xs, atol=1e-8)
    assert np.allclose(sol["z"][:N, nx:], us, atol=1e-8)
    assert np.allclose(sol["z"][N, nx:], 0.0, atol=1e-8)   # u_N decouples


def brute_force_qp(q, soft_rows=()):
    """Exact solution of min 1/2 z'Pz + q'z + sum_soft gamma2/2 xi^2
    s.t. Cz = c, lo <= Gz + xi <= hi (xi only on soft rows) by enumerating every
    (inactive / lower / upper) assignment of the finite-bound rows and keeping the
    one whose equality-constrained KKT solution is primal and dual feasible."""
    P, qv, C, c, G = q["P"].toarray(), q["q"], q["C"].toarray(), q["c"], q["G"].toarray()
    lo, hi, g2 = q["lo"], q["hi"], q["gamma2"]
    nz = P.shape[0]
    soft = list(soft_rows)
    ns = len(soft)
    nw = nz + ns
    H = np.zeros((nw, nw))
    H[:nz, :nz] = P
    for k, r in enumerate(soft):
        H[nz + k, nz + k] = g2[r]
    hv = np.concatenate([qv, np.zeros(ns)])
    Ce = np.hstack([C, np.zeros((C.shape[0], ns))])
    Gw = np.hstack([G, np.zeros((G.shape[0], ns))])
    for k, r in enumerate(soft):
        Gw[r, nz + k] = 1.0
    rows = [i for i in range(G.shape[0]) if np.isfinite(lo[i]) or np.isfinite(hi[i])]
    best = None
    for assign in itertools.product((0, 1, 2), repeat=len(rows)):
        act = [(r, a) for r, a in zip(rows, assign) if a]
        if any((a == 1 and not np.isfinite(lo[r])) or (a == 2 and not np.isfinite(hi[r])) for r, a in act):
            continue
        GA = np.array([Gw[r] for r, _ in act]).reshape(len(act), nw)
        bA = np.array([lo[r] if a == 1 else hi[r] for r, a in act])
        M = np.block([[H, Ce.T, GA.T],
                      [Ce, np.zeros((Ce.shape[0], Ce.shape[0] + len(act)))],
                      [GA, np.zeros((len(act), Ce.shape[0] + len(act)))]])
        rhs = np.concatenate([-hv, c, bA])
        try:
            sol = np.linalg.solve(M, rhs)
        except np.linalg.LinAlgError:
            continue
        wv = sol[:nw]
        yA = sol[nw + Ce.shape[0]:]
        gv = Gw @ wv
        if np.any(gv < lo - 1e-9) or np.any(gv > hi + 1e-9):
            continue
        if any((a == 1 and y > 1e-9) or (a == 2 and y < -1e-9) for (r, a), y in zip(act, yA)):
            continue
        best = wv
        break
    assert best is not None
    return best[:nz], best[nz:]


def test_hard_qp_matches_brute_force():
    p = w.double_integrator(N=2)
    inst = p.instance(0)
    inst["x0"] = np.array([0.5, -0.3, 1.9, -1.8])
    inst["hi"][:, 0:2] = 0.4
    inst["lo"][:, 0:2] = -0.4
    z0 = sqp.rollout(inst)
    q = qpm.build_qp(inst, z0)
    zb, _ = brute_force_qp(q)
    r = admm.admm(q, tight(p.opts), z0.reshape(-1), q["G"] @ z0.reshape(-1),
                  np.zeros(q["C"].shape[0]), np.zeros(q["G"].shape[0]), 0.1)
    assert np.max(np.abs(r["x"] - zb)) < 1e-7
    n_active = np.sum(np.abs(q["G"] @ zb - np.clip(q["G"] @ zb, q["lo"], q["hi"])) < 1e-12)
    assert n_active > 0


def test_soft_qp_matches_brute_force():
    p = w.double_integrator(N=2)
    inst = p.instance(0)
    inst["x0"] = np.array([0.5, -0.3, 2.5, -2.4])        # velocity bounds are violated at t=1
    inst["gamma2"] = np.array([np.inf, np.inf, 3.0, 5.0])  # soften the velocity rows (L2 only)
    inst["gamma1"] = np.zeros(4)
    z0 = sqp.rollout(inst)
    q = qpm.build_qp(inst, z0)
    soft_rows = [i for i in range(q["G"].shape[0]) if np.isfinite(q["gamma2"][i])
                 and (np.isfinite(q["lo"][i]) or np.isfinite(q["hi"][i]))]
    zb, xib = brute_force_qp(q, soft_rows)
    r = admm.admm(q, tight(p.opts), z0.reshape(-1), q["G"] @ z0.reshape(-1),
                  np.zeros(q["C"].shape[0]), np.zeros(q["G"].shape[0]), 0.1)
    assert np.max(np.abs(r["x"] - zb)) < 1e-7
    assert np.max(np.abs(r["xi"][soft_rows] - xib)) < 1e-7
    assert np.max(np.abs(xib)) > 1e-3                      # the slacks are really used
    # invariant of the slack update: gamma2 xi + y_g = 0 on every soft row
    g2 = q["gamma2"]
    m = np.isfinite(g2)
    assert np.max(np.abs(g2[m] * r["xi"][m] + r["yg"][m])) < 1e-9


def paper_smoothed_projection(v, lo, hi, rho, gam):
    """Eq. (proj:tilde) as printed: z = rho/(gam+rho) v + gam/(gam+rho) Pi(v),
    xi = rho/(gam+rho) (Pi(v) - v)."""
    Pi = np.clip(v, lo, hi)
    return rho / (gam + rho) * v + gam / (gam + rho) * Pi, rho / (gam + rho) * (Pi - v)


def test_projection_closed_forms():
    rng = np.random.default_rng(4)
    v = rng.normal(0, 3, 200)
    lo = -np.abs(rng.normal(0, 1, 200))
    hi = np.abs(rng.normal(0, 1, 200))
    rho, gam = 0.7, 2.3
    z, xi = admm.project(v, lo, hi, rho, np.full(200, gam), np.zeros(200))
    zp, xp = paper_smoothed_projection(v, lo, hi, rho, gam)
    assert np.allclose(z, zp) and np.allclose(xi, xp)
    # hard rows and the gamma2 -> inf limit are the plain projection
    zh, xh = admm.project(v, lo, hi, rho, np.full(200, np.inf), np.zeros(200))
    assert np.allclose(zh, np.clip(v, lo, hi)) and np.all(xh == 0)
    zl, _ = admm.project(v, lo, hi, rho, np.full(200, 1e12), np.zeros(200))
    assert np.allclose(zl, np.clip(v, lo, hi), atol=1e-9)
    # with an L1 weight the result minimises the per-row objective (grid search)
    g1 = 0.9
    z1, x1 = admm.project(v[:40], lo[:40], hi[:40], rho, np.full(40, gam), np.full(40, g1))
    for i in range(40):
        xs = np.linspace(-5, 5, 200001)
        # for fixed xi the best z is the clip of v onto [lo - xi, hi - xi]
        zs = np.clip(v[i], lo[i] - xs, hi[i] - xs)
        obj = 0.5 * gam * xs**2 + g1 * np.abs(xs) + 0.5 * rho * (v[i] - zs) ** 2
        k = np.argmin(obj)
        ob = 0.5 * gam * x1[i]**2 + g1 * abs(x1[i]) + 0.5 * rho * (v[i] - z1[i]) ** 2
        assert ob <= obj[k] + 1e-9
        assert abs(xs[k] - x1[i]) < 1e-4


def test_residuals_vanish_at_convergence_and_w_is_zero():
    p = w.racing(B=1, N=8, track_length=100.0)
    inst = p.instance(0)
    z0 = sqp.rollout(inst)
    q = qpm.build_qp(inst, z0)
    r = admm.admm(q, tight(p.opts, iters=40000, eps=1e-10), z0.reshape(-1),
                  q["G"] @ z0.reshape(-1), np.zeros(q["C"].shape[0]), np.zeros(q["G"].shape[0]), 0.1)
    rp, rd, _, _ = admm.residuals(q, r["x"], r["zg"], r["xi"], r["yf"], r["yg"])
    assert rp < 1e-8 and rd < 1e-8
    # soft-row invariant with the L1 term: gamma2 xi + gamma1 sign(xi) + y = 0 or |y| <= gamma1
    rs = admm.slack_dual_residual(r["xi"], r["yg"], q["gamma2"], q["gamma1"])
    assert np.max(np.abs(rs)) < 1e-9
