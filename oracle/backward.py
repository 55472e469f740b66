"""Active-set implicit-differentiation backward pass (Algorithm 2, Section III-D,
Appendix E of the paper), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

1. Active set (Appendix E, "Active constraints identification"): row i is
   lower-active if y_i < -eps_g or (|y_i| < eps_g and g_i + xi_i - lo_i <= eps_g max(1,|lo_i|)),
   upper-active likewise with the upper bound; the dual test takes priority.
   (Readings: the proximity test uses max(1, |bound|) so a zero bound is not
   degenerate, and is applied to the constrained quantity g + xi.)
   A softened row that is active with |xi| > eps_g keeps its slack; an active
   softened row with xi = 0 (held at the L1 kink) behaves as a hard row.
2. The full active-set KKT matrix of Eq. (bwd:slack_adjoint),
       [ H   0        df'  dgA' ] [eta_x ]   [dL/dz ]
       [ 0   gamma2 I 0    E    ] [eta_xi] = [dL/dxi]
       [ df  0        0    0    ] [eta_f ]   [0     ]
       [ dgA E'       0    0    ] [eta_A ]   [0     ]
   is assembled sparse (df includes the initial-state rows) and solved by a
   library LU with partial pivoting.  H is the cost Hessian ("Hessian
   approximation" option) or, with exact_hessian, the Hessian of
   l + y_f'f + y_A'g_A whose constraint curvature is obtained by central
   differences of the analytic Jacobians.
   With `penalty` = gamma_xi, the reduced adjoint QP of Appendix E instead: each
   hard active row is absorbed into the Hessian as the penalty
   gamma_xi/2 (G_A eta_x)^2, i.e. its row of the KKT matrix gets -1/gamma_xi on
   the diagonal of its multiplier (eliminating eta_A = gamma_xi G_A eta_x leaves
   H + gamma_xi G_A'G_A with the dynamics rows as the only constraints); the
   soft active rows keep their exact slack blocks.  The paper notes this
   variant's bias against the exact adjoint; it tends to it as gamma_xi grows.
3. The VJP of Eq. (loss_gradient): grad_theta L = -(dF/dtheta)' eta for
   theta = x_init, diagonal cost weights Q, R, W, references, linear cost
   term, active bounds, and the slack weights (gamma2, gamma1).
Parity: pinned by tests/test_oracle_sqp_backward.py (central finite differences of
the converged FP64 solution map, the gamma closed form, zero gradients of
inactive bounds, and the LQ Riccati adjoint for dL/dx_init).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import models, qp as qp_mod


def active_set(inst, z, xi, yg, eps_g):
    """Boolean masks (lower, upper, slack) [N+1, ng]."""
    g, _ = models.constraints(inst, z)
    val = g + xi
    lo, hi = inst["lo"], inst["hi"]
    with np.errstate(invalid="ignore"):
        lower = np.isfinite(lo) & ((yg < -eps_g) |
                                   ((np.abs(yg) < eps_g) & (val - lo <= eps_g * np.maximum(1.0, np.abs(lo)))))
        upper = (~lower) & np.isfinite(hi) & ((yg > eps_g) |
                                              ((np.abs(yg) < eps_g) & (hi - val <= eps_g * np.maximum(1.0, np.abs(hi)))))
    soft = np.isfinite(inst["gamma2"])[None, :]
    slack = (lower | upper) & soft & (np.abs(xi) > eps_g)
    return lower, upper, slack


def _constraint_curvature(inst, z, yf, yg, active, h=1e-6):
    """d/dz of (df(z)' y_f + dg_A(z)' y_A) by central differences of the analytic
    Jacobians (the curvature part of the Lagrangian Hessian)."""
    nz = z.size
    shape = z.shape
    yA = np.where(active, yg, 0.0)

    def lag_grad(zf):
        zz = zf.reshape(shape)
        q = qp_mod.build_qp(inst, zz)
        return q["C"].T @ yf.reshape(-1) + q["G"].T @ yA.reshape(-1)

    Hc = np.zeros((nz, nz))
    z0 = z.reshape(-1)
    for k in range(nz):
        e = np.zeros(nz)
        e[k] = h
        Hc[:, k] = (lag_grad(z0 + e) - lag_grad(z0 - e)) / (2 * h)
    return 0.5 * (Hc + Hc.T)


def backward(inst, sol, dLdz, dLdxi=None, eps_g=1e-4, exact_hessian=False, penalty=None):
    """Gradients of L with respect to the problem parameters (see module doc).
    sol: dict(z, xi, yf, yg).  penalty: None for the exact active-set adjoint, or
    gamma_xi for the reduced adjoint QP of Appendix E.  Returns (grads dict,
    info dict)."""
    nx, nu, ng, N = inst["nx"], inst["nu"], inst["ng"], inst["N"]
    n = nx + nu
    z, xi, yf, yg = sol["z"], sol["xi"], sol["yf"], sol["yg"]
    if dLdxi is None:
        dLdxi = np.zeros_like(xi)
    q = qp_mod.build_qp(inst, z)
    lower, upper, slack = active_set(inst, z, xi, yg, eps_g)
    active = lower | upper
    act_idx = np.flatnonzero(active.reshape(-1))
    slk_idx = np.flatnonzero(slack.reshape(-1))
    nz = (N + 1) * n
    nf = (N + 1) * nx
    na = act_idx.size
    ns = slk_idx.size

    H = q["P"]
    if exact_hessian:
        H = sp.csr_matrix(H + _constraint_curvature(inst, z, yf, yg, active))
    GA = q["G"][act_idx]
    pos_in_active = {r: k for k, r in enumerate(act_idx)}
    E = sp.csr_matrix((np.ones(ns), (np.arange(ns), [pos_in_active[r] for r in slk_idx])),
                      shape=(ns, na))
    g2 = np.tile(inst["gamma2"], N + 1)[slk_idx]
    K = sp.bmat([[H, None, q["C"].T, GA.T],
                 [None, sp.diags(g2) if ns else None, None, E if ns else None],
                 [q["C"], None, None, None],
                 [GA, E.T if ns else None, None, None]], format="csc") if ns else \
        sp.bmat([[H, q["C"].T, GA.T], [q["C"], None, None], [GA, None, None]], format="csc")
    if penalty is not None:
        # hard active rows (active, no slack) become penalties: -1/gamma_xi on their diagonal
        slack_rows = set(slk_idx.tolist())
        hard = np.array([r not in slack_rows for r in act_idx], dtype=bool)
        d = np.concatenate([np.zeros(nz + ns + nf), np.where(hard, -1.0 / penalty, 0.0)])
        K = (K + sp.diags(d)).tocsc()
    rhs = np.concatenate([dLdz.reshape(-1), dLdxi.reshape(-1)[slk_idx], np.zeros(nf + na)])
    singular = False
    with np.errstate(all="ignore"):
        try:
            eta = spla.spsolve(K, rhs)
        except RuntimeError:        # the LU met an exactly zero pivot: singular, as a non-finite result
            eta = np.full(rhs.shape, np.nan)
    if not np.all(np.isfinite(eta)):
        singular = True
        reg = sp.diags(np.concatenate([np.zeros(nz + ns), -1e-10 * np.ones(nf + na)]))
        eta = spla.spsolve((K + reg).tocsc(), rhs)
    eta_x = eta[:nz].reshape(N + 1, n)
    eta_xi = eta[nz:nz + ns]
    eta_f = eta[nz + ns:nz + ns + nf].reshape(N + 1, nx)
    eta_A = eta[nz + ns + nf:]

    ref = inst["ref"]
    grads = {}
    grads["x0"] = eta_f[0].copy()
    grads["Qd"] = -eta_x[:, :nx] * (z[:, :nx] - ref[:, :nx])
    grads["Rd"] = -eta_x[:, nx:] * (z[:, nx:] - ref[:, nx:])
    grads["ref"] = np.concatenate([inst["Qd"] * eta_x[:, :nx], inst["Rd"] * eta_x[:, nx:]], axis=1)
    grads["lin"] = -eta_x
    du = z[:-1, nx:] - z[1:, nx:]
    de = eta_x[:-1, nx:] - eta_x[1:, nx:]
    grads["Wd"] = -np.sum(de * du, axis=0)
    gA = np.zeros((N + 1) * ng)
    gA[act_idx] = eta_A
    gA = gA.reshape(N + 1, ng)
    grads["lo"] = np.where(lower, gA, 0.0)
    grads["hi"] = np.where(upper, gA, 0.0)
    exi = np.zeros((N + 1) * ng)
    exi[slk_idx] = eta_xi
    exi = exi.reshape(N + 1, ng)
    grads["gamma2"] = -np.sum(xi * exi, axis=0)
    grads["gamma1"] = -np.sum(np.sign(xi) * exi, axis=0)
    info = dict(lower=lower, upper=upper, slack=slack, eta_x=eta_x, eta_f=eta_f,
                eta_A=eta_A, eta_xi=eta_xi, singular=singular)
    return grads, info
