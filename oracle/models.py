"""OCP model functions in FP64: dynamics residuals f_t, inequality functions
g_t, their Jacobians, and the racing centreline.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Dynamics constraints follow Remark A1 of the paper: an explicit model is
f_t = Phi(x_t, u_t) - x_{t+1}; the racing model uses an implicit midpoint
rule f_t = x_t + dt f_c((x_t + x_{t+1})/2, u_t) - x_{t+1}, or the paper's
trapezoidal rule f_t = x_t + dt/2 (f_c(z_t) + f_c(z_{t+1})) - x_{t+1} (both keep
C block-bidiagonal, Remark 2), or the explicit map x_{t+1} = Phi(x_t, u_t)
that 3 Newton steps on the midpoint rule define (Jacobians by the implicit
function theorem).  Jacobians are
returned as the blocks A^-_t = d f_t / d(x_t, u_t) and
A^+_t = d f_t / d(x_{t+1}, u_{t+1}) of Appendix B ("Equality constraints").
All functions act on one instance and are vectorised over stages.
"""
from __future__ import annotations

import math

import numpy as np

from workloads import (BICYCLES, MODEL_BICYCLE, MODEL_BICYCLE_NEWTON, MODEL_BICYCLE_TRAP, MODEL_DI,
                       MODEL_LINEAR, MODEL_QUAD, MODEL_SRB)

NEWTON_MAP_STEPS = 3   # Newton steps that define the explicit map of MODEL_BICYCLE_NEWTON


# ----------------------------------------------------------------------------
# racing centreline: periodic table of (x_c, y_c, psi_c, kappa) every ds metres,
# evaluated by cubic Hermite interpolation of x_c, y_c, psi_c with the knot
# derivatives (cos psi_c, sin psi_c, kappa).
# ----------------------------------------------------------------------------
def track_eval(tab, ds, s):
    """Return (xc, yc, psic, dxc, dyc, dpsic) at arc length(s) s (array)."""
    s = np.asarray(s, dtype=np.float64)
    nt = tab.shape[0] - 1
    L = nt * ds
    sm = s - L * np.floor(s / L)
    k = np.minimum(np.floor(sm / ds).astype(np.int64), nt - 1)
    k = np.maximum(k, 0)
    tau = (sm - k * ds) / ds
    p0 = tab[k, 0:3]
    p1 = tab[k + 1, 0:3]
    m0 = np.stack([np.cos(tab[k, 2]), np.sin(tab[k, 2]), tab[k, 3]], axis=-1)
    m1 = np.stack([np.cos(tab[k + 1, 2]), np.sin(tab[k + 1, 2]), tab[k + 1, 3]], axis=-1)
    t = tau[..., None]
    h00 = 2 * t**3 - 3 * t**2 + 1
    h10 = t**3 - 2 * t**2 + t
    h01 = -2 * t**3 + 3 * t**2
    h11 = t**3 - t**2
    d00 = 6 * t**2 - 6 * t
    d10 = 3 * t**2 - 4 * t + 1
    d01 = -6 * t**2 + 6 * t
    d11 = 3 * t**2 - 2 * t
    p = h00 * p0 + h10 * ds * m0 + h01 * p1 + h11 * ds * m1
    dp = (d00 * p0 + d10 * ds * m0 + d01 * p1 + d11 * ds * m1) / ds
    return p[..., 0], p[..., 1], p[..., 2], dp[..., 0], dp[..., 1], dp[..., 2]


# ----------------------------------------------------------------------------
# continuous-time models
# ----------------------------------------------------------------------------
def bicycle_fc(x, u, dyn, tab):
    """Kinematic bicycle, state (px, py, psi, v, delta, s), control (a, steer rate).
    ds/dt = v cos(psi - psi_c(s)) is the progress along the centreline.
    Returns f_c [T, 6], J_x [T, 6, 6], J_u [T, 6, 2]."""
    L, ds = dyn[1], dyn[2]
    px, py, psi, v, dl, s = (x[:, i] for i in range(6))
    a, w = u[:, 0], u[:, 1]
    _, _, psic, _, _, dpsic = track_eval(tab, ds, s)
    T = x.shape[0]
    c, sn = np.cos(psi), np.sin(psi)
    tn = np.tan(dl)
    dth = psi - psic
    f = np.stack([v * c, v * sn, v * tn / L, a, w, v * np.cos(dth)], axis=1)
    Jx = np.zeros((T, 6, 6))
    Jx[:, 0, 2] = -v * sn
    Jx[:, 0, 3] = c
    Jx[:, 1, 2] = v * c
    Jx[:, 1, 3] = sn
    Jx[:, 2, 3] = tn / L
    Jx[:, 2, 4] = v / (L * np.cos(dl) ** 2)
    Jx[:, 5, 2] = -v * np.sin(dth)
    Jx[:, 5, 3] = np.cos(dth)
    Jx[:, 5, 5] = v * np.sin(dth) * dpsic
    Ju = np.zeros((T, 6, 2))
    Ju[:, 3, 0] = 1.0
    Ju[:, 4, 1] = 1.0
    return f, Jx, Ju


def quad_fc(x, u, dyn):
    """Planar quadrotor, state (px, pz, theta, vx, vz, omega), control (T1, T2)."""
    m, I, arm, g = dyn[1], dyn[2], dyn[3], dyn[4]
    th = x[:, 2]
    Tsum = u[:, 0] + u[:, 1]
    T = x.shape[0]
    f = np.stack([x[:, 3], x[:, 4], x[:, 5], -Tsum * np.sin(th) / m,
                  Tsum * np.cos(th) / m - g, (u[:, 1] - u[:, 0]) * arm / I], axis=1)
    Jx = np.zeros((T, 6, 6))
    Jx[:, 0, 3] = 1.0
    Jx[:, 1, 4] = 1.0
    Jx[:, 2, 5] = 1.0
    Jx[:, 3, 2] = -Tsum * np.cos(th) / m
    Jx[:, 4, 2] = -Tsum * np.sin(th) / m
    Ju = np.zeros((T, 6, 2))
    Ju[:, 3, :] = (-np.sin(th) / m)[:, None]
    Ju[:, 4, :] = (np.cos(th) / m)[:, None]
    Ju[:, 5, 0] = -arm / I
    Ju[:, 5, 1] = arm / I
    return f, Jx, Ju


def quad_rk4(x, u, dyn):
    """Explicit RK4 step of the planar quadrotor with its Jacobians (chain rule
    through the four stages).  Returns Phi [T,6], dPhi/dx [T,6,6], dPhi/du [T,6,2]."""
    dt = dyn[0]
    T = x.shape[0]
    I6 = np.broadcast_to(np.eye(6), (T, 6, 6))
    k1, J1, U1 = quad_fc(x, u, dyn)
    dk1x, dk1u = J1, U1
    x2 = x + 0.5 * dt * k1
    k2, J2, U2 = quad_fc(x2, u, dyn)
    dk2x = J2 @ (I6 + 0.5 * dt * dk1x)
    dk2u = J2 @ (0.5 * dt * dk1u) + U2
    x3 = x + 0.5 * dt * k2
    k3, J3, U3 = quad_fc(x3, u, dyn)
    dk3x = J3 @ (I6 + 0.5 * dt * dk2x)
    dk3u = J3 @ (0.5 * dt * dk2u) + U3
    x4 = x + dt * k3
    k4, J4, U4 = quad_fc(x4, u, dyn)
    dk4x = J4 @ (I6 + dt * dk3x)
    dk4u = J4 @ (dt * dk3u) + U4
    phi = x + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    dphix = I6 + dt / 6.0 * (dk1x + 2 * dk2x + 2 * dk3x + dk4x)
    dphiu = dt / 6.0 * (dk1u + 2 * dk2u + 2 * dk3u + dk4u)
    return phi, dphix, dphiu


def srb_euler_rate_matrix(phi, th):
    """T(Theta) of the ZYX Euler angles (Theta_dot = T omega, omega in the body
    frame; App. humanoid SRB dynamics) and its derivatives with respect to roll
    phi and pitch theta.  Arrays [T, 3, 3]."""
    sp, cp, tt, ct = np.sin(phi), np.cos(phi), np.tan(th), np.cos(th)
    one, zero = np.ones_like(phi), np.zeros_like(phi)
    Tm = np.stack([np.stack([one, sp * tt, cp * tt], -1),
                   np.stack([zero, cp, -sp], -1),
                   np.stack([zero, sp / ct, cp / ct], -1)], -2)
    dphi = np.stack([np.stack([zero, cp * tt, -sp * tt], -1),
                     np.stack([zero, -sp, -cp], -1),
                     np.stack([zero, cp / ct, -sp / ct], -1)], -2)
    sec2 = 1.0 / ct**2
    dth = np.stack([np.stack([zero, sp * sec2, cp * sec2], -1),
                    np.stack([zero, zero, zero], -1),
                    np.stack([zero, sp * tt / ct, cp * tt / ct], -1)], -2)
    return Tm, dphi, dth


def _cross_matrix(r):
    """[r]_x with [r]_x a = r x a; r [..., 3]."""
    z = np.zeros_like(r[..., 0])
    return np.stack([np.stack([z, -r[..., 2], r[..., 1]], -1),
                     np.stack([r[..., 2], z, -r[..., 0]], -1),
                     np.stack([-r[..., 1], r[..., 0], z], -1)], -2)


def srb_fc(x, u, dyn):
    """Single-rigid-body centroidal dynamics (App. humanoid SRB dynamics):
    state (p, Theta, v, omega), control (f_L, f_R) in the world frame,
      p_dot = v,  Theta_dot = T(Theta) omega,  v_dot = (f_L + f_R) / m + g,
      omega_dot = I^-1 (r_L x f_L + r_R x f_R - omega x (I omega)),
    I = diag(Ixx, Iyy, Izz), g = (0, 0, -gravity), the torques as the paper
    writes them.  dyn = [dt, m, Ixx, Iyy, Izz, r_L (3), r_R (3), gravity].
    Returns f [T,12], df/dx [T,12,12], df/du [T,12,6]."""
    m, Id, rL, rR, grav = dyn[1], np.asarray(dyn[2:5]), np.asarray(dyn[5:8]), np.asarray(dyn[8:11]), dyn[11]
    T = x.shape[0]
    Theta, v, w = x[:, 3:6], x[:, 6:9], x[:, 9:12]
    fL, fR = u[:, 0:3], u[:, 3:6]
    Tm, dphi, dth = srb_euler_rate_matrix(Theta[:, 0], Theta[:, 1])
    Iw = w * Id
    tau = np.cross(rL, fL) + np.cross(rR, fR) - np.cross(w, Iw)
    f = np.concatenate([v, np.einsum("tij,tj->ti", Tm, w), (fL + fR) / m + np.array([0.0, 0.0, -grav]), tau / Id], axis=1)
    Jx = np.zeros((T, 12, 12))
    Jx[:, 0:3, 6:9] = np.eye(3)
    Jx[:, 3:6, 3] = np.einsum("tij,tj->ti", dphi, w)
    Jx[:, 3:6, 4] = np.einsum("tij,tj->ti", dth, w)
    Jx[:, 3:6, 9:12] = Tm
    # d(omega x I omega)/d omega = [omega]_x I - [I omega]_x
    Jx[:, 9:12, 9:12] = -(_cross_matrix(w) * Id[None, None, :] - _cross_matrix(Iw)) / Id[None, :, None]
    Ju = np.zeros((T, 12, 6))
    Ju[:, 6:9, 0:3] = np.eye(3) / m
    Ju[:, 6:9, 3:6] = np.eye(3) / m
    Ju[:, 9:12, 0:3] = _cross_matrix(rL) / Id[:, None]
    Ju[:, 9:12, 3:6] = _cross_matrix(rR) / Id[:, None]
    return f, Jx, Ju


def rk4(fc, x, u, dyn):
    """Explicit RK4 step x+ = Phi(x, u) of the continuous dynamics fc (dt =
    dyn[0]) with its Jacobians by the chain rule through the four stages.
    Returns Phi [T,nx], dPhi/dx [T,nx,nx], dPhi/du [T,nx,nu]."""
    dt = dyn[0]
    T, nx = x.shape
    I = np.broadcast_to(np.eye(nx), (T, nx, nx))
    k1, J1, U1 = fc(x, u, dyn)
    k2, J2, U2 = fc(x + 0.5 * dt * k1, u, dyn)
    d2x, d2u = J2 @ (I + 0.5 * dt * J1), J2 @ (0.5 * dt * U1) + U2
    k3, J3, U3 = fc(x + 0.5 * dt * k2, u, dyn)
    d3x, d3u = J3 @ (I + 0.5 * dt * d2x), J3 @ (0.5 * dt * d2u) + U3
    k4, J4, U4 = fc(x + dt * k3, u, dyn)
    d4x, d4u = J4 @ (I + dt * d3x), J4 @ (dt * d3u) + U4
    phi = x + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return phi, I + dt / 6.0 * (J1 + 2 * d2x + 2 * d3x + d4x), dt / 6.0 * (U1 + 2 * d2u + 2 * d3u + d4u)


def di_matrices(dt):
    """Zero-order-hold double integrator in 2-D: position (2), velocity (2)."""
    I2 = np.eye(2)
    A = np.block([[I2, dt * I2], [np.zeros((2, 2)), I2]])
    B = np.vstack([0.5 * dt * dt * I2, dt * I2])
    return A, B


def linear_matrices(inst):
    """A, B and the affine term b of x+ = A x + B u + b (b = 0 when the
    parameters stop after B)."""
    nx, nu = inst["nx"], inst["nu"]
    d = inst["dyn"]
    A = d[:nx * nx].reshape(nx, nx)
    B = d[nx * nx:nx * nx + nx * nu].reshape(nx, nu)
    o = nx * nx + nx * nu
    b = d[o:o + nx].copy() if d.size >= o + nx else np.zeros(nx)
    return A, B, b


# ----------------------------------------------------------------------------
# dynamics residuals f_t and Jacobian blocks (A^-_t, A^+_t), t = 0..N-1
# ----------------------------------------------------------------------------
def dynamics(inst, z):
    """f_t(z_t, z_{t+1}) for t = 0..N-1 and its Jacobian blocks.
    z: [N+1, n].  Returns f [N, nx], Am [N, nx, n], Ap [N, nx, n]."""
    model, nx, nu = inst["model"], inst["nx"], inst["nu"]
    n = nx + nu
    N = z.shape[0] - 1
    x, u = z[:, :nx], z[:, nx:]
    Am = np.zeros((N, nx, n))
    Ap = np.zeros((N, nx, n))
    if model in (MODEL_DI, MODEL_LINEAR, MODEL_QUAD, MODEL_SRB):
        if model == MODEL_QUAD:
            phi, Jx, Ju = quad_rk4(x[:-1], u[:-1], inst["dyn"])
        elif model == MODEL_SRB:
            phi, Jx, Ju = rk4(srb_fc, x[:-1], u[:-1], inst["dyn"])
        else:
            A, B, b = (*di_matrices(inst["dyn"][0]), np.zeros(nx)) if model == MODEL_DI else linear_matrices(inst)
            phi = x[:-1] @ A.T + u[:-1] @ B.T + b
            Jx = np.broadcast_to(A, (N, nx, nx))
            Ju = np.broadcast_to(B, (N, nx, nu))
        f = phi - x[1:]
        Am[:, :, :nx] = Jx
        Am[:, :, nx:] = Ju
        Ap[:, :, :nx] = -np.eye(nx)
        return f, Am, Ap
    if model == MODEL_BICYCLE:
        dt = inst["dyn"][0]
        mid = 0.5 * (x[:-1] + x[1:])
        fc, Jx, Ju = bicycle_fc(mid, u[:-1], inst["dyn"], inst["track"])
        f = x[:-1] + dt * fc - x[1:]
        I = np.eye(nx)
        Am[:, :, :nx] = I + 0.5 * dt * Jx
        Am[:, :, nx:] = dt * Ju
        Ap[:, :, :nx] = -I + 0.5 * dt * Jx
        return f, Am, Ap
    if model == MODEL_BICYCLE_TRAP:
        # Remark A1: f_t = x_t + dt/2 (f_c(x_t, u_t) + f_c(x_{t+1}, u_{t+1})) - x_{t+1}
        dt = inst["dyn"][0]
        fa, Jxa, Jua = bicycle_fc(x[:-1], u[:-1], inst["dyn"], inst["track"])
        fb, Jxb, Jub = bicycle_fc(x[1:], u[1:], inst["dyn"], inst["track"])
        f = x[:-1] + 0.5 * dt * (fa + fb) - x[1:]
        I = np.eye(nx)
        Am[:, :, :nx] = I + 0.5 * dt * Jxa
        Am[:, :, nx:] = 0.5 * dt * Jua
        Ap[:, :, :nx] = -I + 0.5 * dt * Jxb
        Ap[:, :, nx:] = 0.5 * dt * Jub
        return f, Am, Ap
    if model == MODEL_BICYCLE_NEWTON:
        # explicit map Phi(x_t, u_t) - x_{t+1} (Remark A1, explicit form)
        phi, dpx, dpu = newton_map(x[:-1], u[:-1], inst["dyn"], inst["track"])
        f = phi - x[1:]
        Am[:, :, :nx] = dpx
        Am[:, :, nx:] = dpu
        Ap[:, :, :nx] = -np.eye(nx)
        return f, Am, Ap
    raise ValueError(f"unknown model {model}")


def newton_map(x, u, dyn, tab, steps=NEWTON_MAP_STEPS):
    """x+ = Phi(x, u): `steps` Newton steps on the implicit midpoint residual
    r(x+) = x + dt f_c((x + x+)/2, u) - x+ from the explicit Euler step, and its
    Jacobians by the implicit function theorem at the returned x+:
    dPhi/dx = -(dr/dx+)^-1 dr/dx, dPhi/du = -(dr/dx+)^-1 dr/du, with
    dr/dx+ = -I + dt/2 J_x(mid), dr/dx = I + dt/2 J_x(mid), dr/du = dt J_u(mid).
    Vectorised over the first axis of x, u."""
    dt = dyn[0]
    T = x.shape[0]
    I = np.broadcast_to(np.eye(6), (T, 6, 6))
    fc, _, _ = bicycle_fc(x, u, dyn, tab)
    xp = x + dt * fc
    for _ in range(steps):
        fm, Jx, _ = bicycle_fc(0.5 * (x + xp), u, dyn, tab)
        r = x + dt * fm - xp
        xp = xp - np.linalg.solve(-I + 0.5 * dt * Jx, r[..., None])[..., 0]
    _, Jx, Ju = bicycle_fc(0.5 * (x + xp), u, dyn, tab)
    Mp = -I + 0.5 * dt * Jx
    dpx = -np.linalg.solve(Mp, I + 0.5 * dt * Jx)
    dpu = -np.linalg.solve(Mp, dt * Ju)
    return xp, dpx, dpu


def rollout_guess(inst, x, u):
    """Initial guess of x_{t+1} for the Newton rollout: the exact explicit step
    for explicit models, one explicit Euler step for the implicit racing model."""
    model = inst["model"]
    if model == MODEL_QUAD:
        return quad_rk4(x[None], u[None], inst["dyn"])[0][0]
    if model == MODEL_SRB:
        return rk4(srb_fc, x[None], u[None], inst["dyn"])[0][0]
    if model == MODEL_DI:
        A, B = di_matrices(inst["dyn"][0])
        return A @ x + B @ u
    if model == MODEL_LINEAR:
        A, B, b = linear_matrices(inst)
        return A @ x + B @ u + b
    if model in (MODEL_BICYCLE, MODEL_BICYCLE_TRAP):
        fc, _, _ = bicycle_fc(x[None], u[None], inst["dyn"], inst["track"])
        return x + inst["dyn"][0] * fc[0]
    if model == MODEL_BICYCLE_NEWTON:
        return newton_map(x[None], u[None], inst["dyn"], inst["track"])[0][0]
    raise ValueError(model)


# ----------------------------------------------------------------------------
# inequality functions g_t(z_t) and Jacobians G_t, t = 0..N
# ----------------------------------------------------------------------------
def constraints(inst, z):
    """g_t(z_t) [N+1, ng] and G_t = dg_t/dz_t [N+1, ng, n]."""
    model, nx, nu, ng = inst["model"], inst["nx"], inst["nu"], inst["ng"]
    n = nx + nu
    T = z.shape[0]
    G = np.zeros((T, ng, n))
    if model == MODEL_DI:
        # rows: u1, u2, vx, vy
        g = np.stack([z[:, 4], z[:, 5], z[:, 2], z[:, 3]], axis=1)
        G[:, 0, 4] = G[:, 1, 5] = G[:, 2, 2] = G[:, 3, 3] = 1.0
        return g, G
    if model in (MODEL_LINEAR, MODEL_SRB):
        # rows: the controls (box constraints; SRB: the friction cone as a box on the foot forces)
        g = z[:, nx:nx + ng].copy()
        for i in range(ng):
            G[:, i, nx + i] = 1.0
        return g, G
    if model == MODEL_QUAD:
        g = z[:, 6:8].copy()
        G[:, 0, 6] = G[:, 1, 7] = 1.0
        return g, G
    if model in BICYCLES:
        # rows: accel, steer rate, speed, steering angle, lateral error e(px, py, s)
        tab, dsk = inst["track"], inst["dyn"][2]
        px, py, s = z[:, 0], z[:, 1], z[:, 5]
        xc, yc, psic, dxc, dyc, dpsic = track_eval(tab, dsk, s)
        sp, cp = np.sin(psic), np.cos(psic)
        e = -(px - xc) * sp + (py - yc) * cp
        de_ds = dxc * sp - dyc * cp - dpsic * ((px - xc) * cp + (py - yc) * sp)
        g = np.stack([z[:, 6], z[:, 7], z[:, 3], z[:, 4], e], axis=1)
        G[:, 0, 6] = G[:, 1, 7] = G[:, 2, 3] = G[:, 3, 4] = 1.0
        G[:, 4, 0] = -sp
        G[:, 4, 1] = cp
        G[:, 4, 5] = de_ds
        return g, G
    raise ValueError(model)


def selector_rows(inst):
    """For each constraint row r of g_t, the index j of the stage variable it
    bounds directly (g_t,r = z_t,j, as `constraints` defines the row), or -1
    for a row that is a function of several variables (the bicycle's lateral
    error).  Used by the rescaling of the QP (Remark 4) to divide a box row by
    its variable's scale."""
    model, nx, ng = inst["model"], inst["nx"], inst["ng"]
    if model == MODEL_DI:
        return np.array([4, 5, 2, 3])
    if model in (MODEL_LINEAR, MODEL_SRB):
        return np.arange(nx, nx + ng)
    if model == MODEL_QUAD:
        return np.array([6, 7])
    if model in BICYCLES:
        return np.array([6, 7, 3, 4, -1])
    raise ValueError(model)


# ----------------------------------------------------------------------------
# cost (diagonal quadratic + control rate + linear term)
# ----------------------------------------------------------------------------
def cost(inst, z):
    """Total stage + terminal cost of the OCP (without slack penalties)."""
    nx = inst["nx"]
    dx = z[:, :nx] - inst["ref"][:, :nx]
    du = z[:, nx:] - inst["ref"][:, nx:]
    val = 0.5 * np.sum(inst["Qd"] * dx * dx) + 0.5 * np.sum(inst["Rd"] * du * du)
    du_rate = z[:-1, nx:] - z[1:, nx:]
    val += 0.5 * np.sum(inst["Wd"][None, :] * du_rate * du_rate)
    val += np.sum(inst["lin"] * z)
    return float(val)


def cost_grad(inst, z):
    nx = inst["nx"]
    gr = np.zeros_like(z)
    gr[:, :nx] = inst["Qd"] * (z[:, :nx] - inst["ref"][:, :nx])
    gr[:, nx:] = inst["Rd"] * (z[:, nx:] - inst["ref"][:, nx:])
    d = inst["Wd"][None, :] * (z[:-1, nx:] - z[1:, nx:])
    gr[:-1, nx:] += d
    gr[1:, nx:] -= d
    gr += inst["lin"]
    return gr


def slack_cost(inst, xi):
    """gamma2/2 xi^2 + gamma1 |xi| over the softened rows (hard rows carry no xi)."""
    g2, g1 = inst["gamma2"], inst["gamma1"]
    soft = np.isfinite(g2)
    if not np.any(soft):
        return 0.0
    x = xi[:, soft]
    return float(np.sum(0.5 * g2[soft][None, :] * x * x + g1[soft][None, :] * np.abs(x)))
