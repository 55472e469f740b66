"""QP approximation of the OCP at an SQP iterate, in FP64 (Section III-A and
Appendix B of the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The global matrices are assembled exactly as Appendix B writes them:
  P: block-tridiagonal, D_0 = H^-_0, D_t = H^+_{t-1} + H^-_t, off-diagonal
     blocks from H^{+-}_t (the (t, t+1) block is H^{+-}_t, the (t+1, t) block
     its transpose);
  q: q_0 = q^-_0, q_t = q^+_{t-1} + q^-_t  (gradients at the iterate);
  C: rows [A_init; A^-_t, A^+_t], c = (x_init, b_0, ..., b_{N-1}) with
     b_t = A^-_t zbar_t + A^+_t zbar_{t+1} - f_t(zbar);
  G: block-diagonal G_t = dg_t/dz_t with shifted bounds
     lo_t - g_t(zbar) + G_t zbar_t,  hi_t - g_t(zbar) + G_t zbar_t.
The QP variable is the absolute stage vector (the constraints are written for
the absolute point), so the linear term used by the QP is
q_abs = q - P zbar: the model of the cost is
l(zbar) + q'(z - zbar) + 1/2 (z - zbar)' P (z - zbar).
Parity: pinned by tests/test_oracle_admm.py and tests/test_oracle_models.py
(dense S identity, exact QP model of a quadratic cost, Jacobians vs
finite differences).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import models


def stage_cost_blocks(inst, z):
    """Per-stage derivatives of the cost at z (Appendix B, "Cost"):
    Hm[t] = d2 l_t / dz_t^2, Hp[t] = d2 l_t / dz_{t+1}^2, Hpm[t] = d2 l_t / dz_t dz_{t+1}
    (t < N), qm[t] = dl_t/dz_t, qp[t] = dl_t/dz_{t+1}; the terminal cost gives
    Hm[N], qm[N]."""
    nx, nu = inst["nx"], inst["nu"]
    n = nx + nu
    N = z.shape[0] - 1
    Q, R, W = inst["Qd"], inst["Rd"], inst["Wd"]
    ref, lin = inst["ref"], inst["lin"]
    Hm = np.zeros((N + 1, n, n))
    Hp = np.zeros((N, n, n))
    Hpm = np.zeros((N, n, n))
    qm = np.zeros((N + 1, n))
    qp = np.zeros((N, n))
    for t in range(N + 1):
        Hm[t, :nx, :nx] = np.diag(Q[t])
        Hm[t, nx:, nx:] = np.diag(R[t])
        qm[t, :nx] = Q[t] * (z[t, :nx] - ref[t, :nx])
        qm[t, nx:] = R[t] * (z[t, nx:] - ref[t, nx:])
        qm[t] += lin[t]
        if t < N:
            # control-rate term 1/2 (u_t - u_{t+1})' W (u_t - u_{t+1})
            Hm[t, nx:, nx:] += np.diag(W)
            Hp[t, nx:, nx:] = np.diag(W)
            Hpm[t, nx:, nx:] = -np.diag(W)
            d = W * (z[t, nx:] - z[t + 1, nx:])
            qm[t, nx:] += d
            qp[t, nx:] = -d
    return Hm, Hp, Hpm, qm, qp


def _place(shape, groups):
    """Sparse matrix whose dense blocks blocks[t] sit at (row0[t], col0[t])."""
    rows, cols, vals = [], [], []
    for blocks, r0, c0 in groups:
        T, a, b = blocks.shape
        ii, jj = np.meshgrid(np.arange(a), np.arange(b), indexing="ij")
        rows.append((r0[:, None, None] + ii[None]).reshape(-1))
        cols.append((c0[:, None, None] + jj[None]).reshape(-1))
        vals.append(blocks.reshape(-1))
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    keep = vals != 0.0
    return sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=shape)


def build_qp(inst, zbar):
    """Assemble the QP at the iterate zbar [N+1, n].  Returns a dict with the
    global sparse matrices and the per-stage blocks used to build them."""
    nx, nu, ng = inst["nx"], inst["nu"], inst["ng"]
    n = nx + nu
    N = zbar.shape[0] - 1
    nz = (N + 1) * n

    Hm, Hp, Hpm, qm, qp = stage_cost_blocks(inst, zbar)
    D = Hm.copy()
    D[1:] += Hp
    t_all = np.arange(N + 1)
    t_off = np.arange(N)
    P = _place((nz, nz), [(D, t_all * n, t_all * n),
                          (Hpm, t_off * n, (t_off + 1) * n),
                          (np.transpose(Hpm, (0, 2, 1)), (t_off + 1) * n, t_off * n)])
    qv = qm.copy()
    qv[1:] += qp
    q_abs = qv.reshape(-1) - P @ zbar.reshape(-1)

    f, Am, Ap = models.dynamics(inst, zbar)
    Ainit = np.zeros((1, nx, n))
    Ainit[0, :, :nx] = np.eye(nx)
    C = _place((nx * (N + 1), nz), [(Ainit, np.array([0]), np.array([0])),
                                    (Am, (t_off + 1) * nx, t_off * n),
                                    (Ap, (t_off + 1) * nx, (t_off + 1) * n)])
    b = np.einsum("tij,tj->ti", Am, zbar[:-1]) + np.einsum("tij,tj->ti", Ap, zbar[1:]) - f
    c = np.concatenate([inst["x0"], b.reshape(-1)])

    g, Gt = models.constraints(inst, zbar)
    Gz = np.einsum("tij,tj->ti", Gt, zbar)
    G = _place((ng * (N + 1), nz), [(Gt, t_all * ng, t_all * n)])
    lo = (inst["lo"] - g + Gz).reshape(-1)
    hi = (inst["hi"] - g + Gz).reshape(-1)

    gam2 = np.tile(inst["gamma2"], N + 1)
    gam1 = np.tile(inst["gamma1"], N + 1)
    assert P.shape == (nz, nz) and C.shape == (nx * (N + 1), nz) and G.shape == (ng * (N + 1), nz)
    return dict(P=P, q=q_abs, C=C, c=c, G=G, lo=lo, hi=hi, gamma2=gam2, gamma1=gam1,
                D=D, E=Hpm, Am=Am, Ap=Ap, Gt=Gt, f=f, g=g, N=N, nx=nx, nu=nu, ng=ng, n=n)


def schur_blocks(qp, sigma, rho_f, rho_g):
    """Theta_t and Phi_t of Appendix C ("Structure from OCP"), written from the
    block formulas.  Used only by the tests to pin the identity
    S = P + sigma I + rho_f C'C + rho_g G'G of the assembled matrices;
    Phi_t is the (t+1, t) block of S."""
    N, n, nx = qp["N"], qp["n"], qp["nx"]
    D, E, Am, Ap, Gt = qp["D"], qp["E"], qp["Am"], qp["Ap"], qp["Gt"]
    Ainit = np.zeros((nx, n))
    Ainit[:, :nx] = np.eye(nx)
    Th = np.zeros((N + 1, n, n))
    Ph = np.zeros((N, n, n))
    for t in range(N + 1):
        Th[t] = D[t] + sigma * np.eye(n) + rho_g * Gt[t].T @ Gt[t]
        if t == 0:
            Th[t] += rho_f * Ainit.T @ Ainit
        if t >= 1:
            Th[t] += rho_f * Ap[t - 1].T @ Ap[t - 1]
        if t < N:
            Th[t] += rho_f * Am[t].T @ Am[t]
    for t in range(N):
        Ph[t] = E[t].T + rho_f * Ap[t].T @ Am[t]
    return Th, Ph
