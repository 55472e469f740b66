"""ADMM QP solver of the paper (Algorithm 3, Section III-B, Appendix C), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

One iteration, in the paper's order (z_f is never stored: z_f = c):
  eta   = sigma x - q + C'(rho_f c - y_f) + G'(rho_g z_g - y_g)     (Eq. admm:schur)
  xt    = S^{-1} eta,   S = P + sigma I + rho_f C'C + rho_g G'G
  zt_f  = C xt,  zt_g = G xt
  x     = alpha xt + (1-alpha) x                                      (over-relaxation)
  zh_f  = alpha zt_f + (1-alpha) c,  zh_g = alpha zt_g + (1-alpha) z_g
  v     = zh_g + y_g / rho_g
  z_g, xi = projection of v (hard rows), smoothed projection (soft rows)
  y_f  += rho_f (zh_f - c),  y_g += rho_g (zh_g - z_g)
then the residuals of Eq. (admm:residuals), the termination test of
Eq. (admm:termination:slack) and, every k_rho_iter iterations, the rho rule of
Eq. (rho:update) with refactorisation when a new rho is accepted.

S is formed from the assembled sparse matrices (the plain definition) and
factored by a library banded Cholesky; no block-tridiagonal formulas are used
here.  The slack rows use the per-row L1+L2 penalty gamma2/2 xi^2 + gamma1 |xi|;
with gamma1 = 0 the projection is exactly the smoothed projection of
Eq. (proj:tilde), and gamma2 = inf makes the row hard.
Parity: pinned by tests/test_oracle_admm.py (closed-form Riccati solution of
the unconstrained LQ problem, brute-force active-set enumeration of tiny QPs,
the slack closed form, invariants w = 0 / gamma xi + y = 0, KKT residuals).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def project(v, lo, hi, rho_g, gamma2, gamma1):
    """Minimiser over (z, xi) of gamma2/2 xi^2 + gamma1 |xi| + I_[lo,hi](z + xi)
    + rho_g/2 (v - z)^2, row by row.  Hard rows (gamma2 = inf): z = clip(v), xi = 0.
    Soft rows above the upper bound: s = max(0, (rho_g (v-hi) - gamma1)/(rho_g+gamma2)),
    z = hi + s, xi = -s; symmetric below the lower bound; inside: z = v, xi = 0."""
    z = np.clip(v, lo, hi)
    xi = np.zeros_like(v)
    soft = np.isfinite(gamma2)
    if np.any(soft):
        vs, los, his = v[soft], lo[soft], hi[soft]
        g2, g1 = gamma2[soft], gamma1[soft]
        zs = vs.copy()
        xs = np.zeros_like(vs)
        up = vs > his
        s_up = np.maximum(0.0, (rho_g * (vs - his) - g1) / (rho_g + g2))
        zs[up] = his[up] + s_up[up]
        xs[up] = -s_up[up]
        dn = vs < los
        s_dn = np.maximum(0.0, (rho_g * (los - vs) - g1) / (rho_g + g2))
        zs[dn] = los[dn] - s_dn[dn]
        xs[dn] = s_dn[dn]
        z[soft] = zs
        xi[soft] = xs
    return z, xi


def slack_dual_residual(xi, yg, gamma2, gamma1):
    """Second block of r_dual for the soft rows: d/dxi (gamma2/2 xi^2 + gamma1|xi|) + y_g,
    i.e. gamma2 xi + gamma1 sign(xi) + y_g when xi != 0 and the distance of -y_g to
    [-gamma1, gamma1] when xi = 0 (subgradient at the kink)."""
    soft = np.isfinite(gamma2)
    r = np.zeros(int(np.count_nonzero(soft)))
    x, y, g2, g1 = xi[soft], yg[soft], gamma2[soft], gamma1[soft]
    nz = x != 0.0
    r[nz] = g2[nz] * x[nz] + g1[nz] * np.sign(x[nz]) + y[nz]
    r[~nz] = np.maximum(0.0, np.abs(y[~nz]) - g1[~nz])
    return r


def residuals(qp, x, zg, xi, yf, yg):
    """(r_prim, r_dual, prim_norm, dual_norm) of Eq. (admm:residuals) and the
    normalisers of Eq. (admm:termination:slack)."""
    P, q, C, c, G = qp["P"], qp["q"], qp["C"], qp["c"], qp["G"]
    g2, g1 = qp["gamma2"], qp["gamma1"]
    Cx, Gx = C @ x, G @ x
    r_prim = max(_ninf(Cx - c), _ninf(Gx - zg))
    Px = P @ x
    Aty = C.T @ yf + G.T @ yg
    rs = slack_dual_residual(xi, yg, g2, g1)
    r_dual = max(_ninf(Px + q + Aty), _ninf(rs))
    soft = np.isfinite(g2)
    prim_norm = max(_ninf(Cx), _ninf(Gx), _ninf(c), _ninf(zg))
    dual_norm = max(_ninf(Px), _ninf(Aty), _ninf(q), _ninf(g2[soft] * xi[soft]), _ninf(yg[soft]))
    return r_prim, r_dual, prim_norm, dual_norm


def _ninf(v):
    return float(np.max(np.abs(v))) if v.size else 0.0


class _BandedSPD:
    """Banded Cholesky factorisation of a sparse SPD matrix (library routine)."""

    def __init__(self, S):
        S = sp.coo_matrix(sp.triu(S))
        u = int(np.max(S.col - S.row)) if S.nnz else 0
        n = S.shape[0]
        ab = np.zeros((u + 1, n))
        ab[u + S.row - S.col, S.col] = S.data
        self.cb = sla.cholesky_banded(ab, lower=False)

    def solve(self, b):
        return sla.cho_solve_banded((self.cb, False), b)


def form_S(qp, sigma, rho_f, rho_g):
    nz = qp["P"].shape[0]
    C, G = qp["C"], qp["G"]
    return (qp["P"] + sigma * sp.identity(nz) + rho_f * (C.T @ C) + rho_g * (G.T @ G)).tocsr()


def admm(qp, opts, x, zg, yf, yg, rho_bar, rho_schedule=None, perturb_S=None):
    """Run Algorithm 3 from the warm start (x, z_g, y_f, y_g) with rho_bar.

    rho_schedule: optional dict {iteration: rho_bar} that replaces the adaptive
    rule (used only to replay another solver's accepted rho values).
    perturb_S: optional callable applied to S before each factorisation (used
    only to measure how the fixed-count result responds to a backward error of
    the factorisation, as a lower-precision solver incurs); None = exact S.
    Returns dict(x, zg, xi, yf, yg, rho_bar, iters, r_prim, r_dual, refactors,
    converged, rho_events)."""
    sigma, alpha = opts.sigma, opts.alpha
    q, C, c, G, lo, hi = qp["q"], qp["C"], qp["c"], qp["G"], qp["lo"], qp["hi"]
    g2, g1 = qp["gamma2"], qp["gamma1"]
    x, zg, yf, yg = x.copy(), zg.copy(), yf.copy(), yg.copy()
    xi = np.zeros_like(zg)

    def factor(rb):
        S = form_S(qp, sigma, 1e3 * rb, rb)
        return _BandedSPD(S if perturb_S is None else perturb_S(S))

    F = factor(rho_bar)
    refactors = 1
    rho_events = []
    converged = False
    r_prim = r_dual = math.inf
    pn = dn = 0.0
    k = 0
    for k in range(1, opts.max_admm + 1):
        rho_f, rho_g = 1e3 * rho_bar, rho_bar
        eta = sigma * x - q + C.T @ (rho_f * c - yf) + G.T @ (rho_g * zg - yg)
        xt = F.solve(eta)
        ztf = C @ xt
        ztg = G @ xt
        x = alpha * xt + (1.0 - alpha) * x
        zhf = alpha * ztf + (1.0 - alpha) * c
        zhg = alpha * ztg + (1.0 - alpha) * zg
        v = zhg + yg / rho_g
        zg_new, xi = project(v, lo, hi, rho_g, g2, g1)
        yf = yf + rho_f * (zhf - c)
        yg = yg + rho_g * (zhg - zg_new)
        zg = zg_new

        check_conv = opts.early_exit and (k % opts.check_every == 0)
        check_rho = (k % opts.k_rho_iter == 0) and k < opts.max_admm
        if check_conv or check_rho or k == opts.max_admm:
            r_prim, r_dual, pn, dn = residuals(qp, x, zg, xi, yf, yg)
            converged = (r_prim <= opts.eps_abs + opts.eps_rel * pn and
                         r_dual <= opts.eps_abs + opts.eps_rel * dn)
            if check_conv and converged:
                break
            if check_rho:
                if rho_schedule is not None:
                    new = rho_schedule.get(k)
                    if new is not None and new != rho_bar:
                        rho_bar = new
                        F = factor(rho_bar)
                        refactors += 1
                        rho_events.append((k, rho_bar))
                elif r_dual > 0.0 and not converged:
                    ratio = (r_prim / max(pn, 1e-30)) / max(r_dual / max(dn, 1e-30), 1e-30)
                    cand = min(max(rho_bar * math.sqrt(ratio), opts.rho_min), opts.rho_max)
                    if max(cand / rho_bar, rho_bar / cand) > opts.k_rho_ratio:
                        rho_bar = cand
                        F = factor(rho_bar)
                        refactors += 1
                        rho_events.append((k, rho_bar))
    return dict(x=x, zg=zg, xi=xi, yf=yf, yg=yg, rho_bar=rho_bar, iters=k,
                r_prim=r_prim, r_dual=r_dual, prim_norm=pn, dual_norm=dn, refactors=refactors,
                converged=converged, rho_events=rho_events)


def pow2_floor(s):
    """Largest power of two not above s > 0, taken from the FP32 value of s
    (s = m 2^e with m in [0.5, 1) gives 2^(e-1)).  Scaling by powers of two is
    exact in binary floating point, so the scaled QP carries no rounding of its
    own.  An entry that is not positive and finite counts as 1."""
    s32 = np.asarray(s, dtype=np.float32).astype(np.float64)
    ok = np.isfinite(s32) & (s32 > 0.0)
    _, e = np.frexp(np.where(ok, s32, 1.0))
    return np.where(ok, np.ldexp(1.0, e - 1), 1.0)


def rescale_qp(qp, d, sel):
    """The QP after the change of variables z = D zh that normalises the states
    and controls (Remark 4, Section III-B).  The paper gives no recipe; the
    reading built here:
      D = diag(d) on every stage (d = pow2_floor of the caller's scales, one
          per state and control component),
      the dynamics rows (initial condition included) are divided by the scale
          of the state component they define, E_f = D_x^-1 per stage, so that
          A^+ = [-I 0] stays a unit block,
      a row of g that bounds one variable z_j directly (sel[r] = j) is divided
          by d_j (it stays a unit selector), any other row is left as it is.
    With Sigma = diag(D, E_f, E_g) the scaled data are P^ = D P D, q^ = D q,
    C^ = E_f C D, c^ = E_f c, G^ = E_g G D, bounds E_g lo, E_g hi, and the slack
    penalty of row r in scaled units gamma2 / e_r^2, gamma1 / e_r.
    Returns (scaled qp, Dv, Ef, Eg): the diagonal scales of every variable,
    dynamics row and constraint row."""
    N, n, nx, ng = qp["N"], qp["n"], qp["nx"], qp["ng"]
    d = pow2_floor(d)
    Dv = np.tile(d, N + 1)
    Ef = 1.0 / np.tile(d[:nx], N + 1)
    er = np.array([1.0 / d[j] if j >= 0 else 1.0 for j in sel])
    Eg = np.tile(er, N + 1)
    Dm, Efm, Egm = sp.diags(Dv), sp.diags(Ef), sp.diags(Eg)
    out = dict(qp)
    out.update(P=(Dm @ qp["P"] @ Dm).tocsr(), q=Dv * qp["q"],
               C=(Efm @ qp["C"] @ Dm).tocsr(), c=Ef * qp["c"],
               G=(Egm @ qp["G"] @ Dm).tocsr(), lo=Eg * qp["lo"], hi=Eg * qp["hi"],
               gamma2=qp["gamma2"] / Eg ** 2, gamma1=qp["gamma1"] / Eg)
    return out, Dv, Ef, Eg


def admm_rescaled(qp, opts, d, sel, x, zg, yf, yg, rho_bar, **kw):
    """Algorithm 3 run on the rescaled QP of `rescale_qp`, from the warm start
    mapped into scaled units (xh = D^-1 x, zh_g = E_g z_g, yh_f = E_f^-1 y_f,
    yh_g = E_g^-1 y_g), with its results mapped back (x = D xh, z_g = E_g^-1 zh_g,
    xi = E_g^-1 xih, y_f = E_f yh_f, y_g = E_g yh_g).  rho, the residuals, the
    termination test and the rho rule all act in scaled units; the returned
    residuals are the scaled ones.  Parity: pinned by tests/test_oracle_rescale.py
    (invariance of the converged solution and multipliers, unit scales, and a
    uniform scale equal to a scaled cost at a fixed count)."""
    sq, Dv, Ef, Eg = rescale_qp(qp, d, sel)
    res = admm(sq, opts, x / Dv, Eg * zg, yf / Ef, yg / Eg, rho_bar, **kw)
    res = dict(res)
    res.update(x=Dv * res["x"], zg=res["zg"] / Eg, xi=res["xi"] / Eg, yf=Ef * res["yf"], yg=Eg * res["yg"])
    return res
