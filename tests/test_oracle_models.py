"""Pins of the oracle's model functions: analytic Jacobians against central
finite differences, centreline interpolation continuity, the Newton rollout."""
import numpy as np
import pytest

import workloads as w
from oracle import models, sqp


def _fd_jac(fun, x, h=1e-6):
    f0 = fun(x)
    J = np.zeros((f0.size, x.size))
    for k in range(x.size):
        e = np.zeros_like(x)
        e[k] = h
        J[:, k] = (fun(x + e) - fun(x - e)).reshape(-1) / (2 * h)
    return J


def _instances():
    out = []
    p = w.double_integrator(N=4)
    out.append(p.instance(0))
    for integ in ("midpoint", "trapezoidal", "newton_map"):
        p = w.racing(B=1, N=4, track_length=100.0, integrator=integ)
        out.append(p.instance(0))
    p = w.tracking(B=1, nx=5, nu=3, N=4)
    out.append(p.instance(0))
    p = w.humanoid(B=1, N=4)
    out.append(p.instance(0))
    p = w.uneven(B=8, N_lo=4, N_hi=6, seed=3)
    for i in range(8):
        if p.model[i] == w.MODEL_QUAD:
            out.append(p.instance(i))
            break
    return out


@pytest.mark.parametrize("inst", _instances(), ids=lambda d: w.MODEL_NAMES[d["model"]])
def test_dynamics_and_constraint_jacobians(inst):
    rng = np.random.default_rng(0)
    nx, nu, N = inst["nx"], inst["nu"], inst["N"]
    z = rng.normal(0, 1, (N + 1, nx + nu))
    if inst["model"] in w.BICYCLES:
        z[:, 3] = 10 + rng.uniform(0, 5, N + 1)      # speed
        z[:, 4] *= 0.2                                # steering angle
        z[:, 5] = 3.0 + np.arange(N + 1) * 0.7 + 0.13  # progress, off the knots
    f, Am, Ap = models.dynamics(inst, z)
    for t in range(N):
        def ft(v, t=t):
            zz = z.copy()
            zz[t] = v[:nx + nu]
            zz[t + 1] = v[nx + nu:]
            return models.dynamics(inst, zz)[0][t]
        J = _fd_jac(ft, np.concatenate([z[t], z[t + 1]]))
        # (the Newton map's Jacobian comes from the implicit function theorem at the
        # 3-step Newton point; it matches the map's own derivative to the Newton residual)
        assert np.allclose(J[:, :nx + nu], Am[t], atol=1e-6, rtol=1e-6)
        assert np.allclose(J[:, nx + nu:], Ap[t], atol=1e-6, rtol=1e-6)
    g, G = models.constraints(inst, z)
    for t in range(N + 1):
        def gt(v, t=t):
            zz = z.copy()
            zz[t] = v
            return models.constraints(inst, zz)[0][t]
        J = _fd_jac(gt, z[t].copy())
        assert np.allclose(J, G[t], atol=1e-6, rtol=1e-6)


def test_track_interpolation_is_c1_and_periodic():
    rng = np.random.default_rng(1)
    tab = w.closed_track(rng, length=400.0)
    ds = w.TRACK_DS
    nt = tab.shape[0] - 1
    # knots reproduce the table, derivatives match the tabulated tangents
    s = np.arange(nt) * ds
    xc, yc, psic, dxc, dyc, dpsic = models.track_eval(tab, ds, s)
    assert np.allclose(xc, tab[:-1, 0]) and np.allclose(yc, tab[:-1, 1])
    assert np.allclose(dxc, np.cos(tab[:-1, 2])) and np.allclose(dpsic, tab[:-1, 3])
    # continuity across knots (left/right limits) and across the periodic seam
    eps = 1e-9
    for sk in [ds * 7, ds * (nt - 1), nt * ds]:
        a = np.array(models.track_eval(tab, ds, sk - eps))
        b = np.array(models.track_eval(tab, ds, sk + eps))
        a[2] = np.mod(a[2], 2 * np.pi)
        b[2] = np.mod(b[2], 2 * np.pi)
        assert np.allclose(a, b, atol=1e-6)
    # derivative of the position is the analytic one
    sq = np.array([3.3, 101.7, 250.2])
    h = 1e-6
    xp = models.track_eval(tab, ds, sq + h)
    xm = models.track_eval(tab, ds, sq - h)
    d = models.track_eval(tab, ds, sq)
    for k in range(3):
        assert np.allclose((xp[k] - xm[k]) / (2 * h), d[3 + k], atol=1e-5)


def test_newton_rollout_satisfies_dynamics():
    p = w.racing(B=1, N=20, track_length=200.0)
    inst = p.instance(0)
    z = sqp.rollout(inst, newton_steps=3)
    f, _, _ = models.dynamics(inst, z)
    assert np.max(np.abs(f)) < 1e-9
    p = w.uneven(B=16, N_lo=8, N_hi=12, seed=5)
    for i in range(16):
        inst = p.instance(i)
        z = sqp.rollout(inst, newton_steps=3)
        f, _, _ = models.dynamics(inst, z)
        assert np.max(np.abs(f)) < 1e-9


def test_newton_map_is_the_midpoint_solution():
    """The explicit map of the Newton-map variant: 3 Newton steps from the explicit
    Euler step solve the implicit midpoint equation to rounding (quadratic
    convergence on a smooth motion), so it equals a 30-step Newton solve, and its
    IFT Jacobian equals the central-difference derivative of that solution."""
    p = w.racing(B=1, N=4, track_length=100.0, integrator="newton_map")
    inst = p.instance(0)
    rng = np.random.default_rng(2)
    x = np.array([[3.0, 1.0, 0.2, 11.0, 0.05, 4.1]])
    u = np.array([[0.8, -0.3]])
    phi, dpx, dpu = models.newton_map(x, u, inst["dyn"], inst["track"])
    ref, _, _ = models.newton_map(x, u, inst["dyn"], inst["track"], steps=30)
    assert np.max(np.abs(phi - ref)) < 1e-12
    dt = inst["dyn"][0]
    fm, _, _ = models.bicycle_fc(0.5 * (x + phi), u, inst["dyn"], inst["track"])
    assert np.max(np.abs(x + dt * fm - phi)) < 1e-12          # midpoint residual
    J = _fd_jac(lambda v: models.newton_map(v[None, :6], v[None, 6:], inst["dyn"], inst["track"], steps=30)[0][0],
                np.concatenate([x[0], u[0]]))
    assert np.allclose(J[:, :6], dpx[0], atol=1e-7) and np.allclose(J[:, 6:], dpu[0], atol=1e-7)


def test_trapezoidal_rule_is_exact_for_uniform_motion():
    """x_{t+1} = x_t + dt/2 (f_c(z_t) + f_c(z_{t+1})) holds exactly for a straight
    line at constant speed on a straight track aligned with it (f_c is constant
    along that motion)."""
    s = np.arange(0.0, 200.25, w.TRACK_DS)
    tab = np.stack([s * np.cos(0.3), s * np.sin(0.3), np.full_like(s, 0.3), np.zeros_like(s)], 1)
    dyn = np.array([0.05, 2.7, w.TRACK_DS, float(len(s) - 1)])
    v, dt = 8.0, 0.05
    z = np.zeros((5, 8))
    for t in range(5):
        q = 5.0 + v * dt * t
        z[t, :6] = [q * np.cos(0.3), q * np.sin(0.3), 0.3, v, 0.0, q]
    inst = dict(model=w.MODEL_BICYCLE_TRAP, nx=6, nu=2, dyn=dyn, track=tab)
    f, _, _ = models.dynamics(inst, z)
    assert np.max(np.abs(f)) < 1e-12


# ----------------------------------------------------------------------------
# single-rigid-body humanoid (App. humanoid SRB dynamics): closed-form motions
# ----------------------------------------------------------------------------
def _srb_dyn():
    return w.humanoid(B=1).dyn[0]


def test_srb_standing_balance_is_an_equilibrium():
    """Feet below the CoM in x, each carrying half the weight, at rest and level:
    the net force and the net torque vanish, so every rate is zero."""
    d = _srb_dyn()
    m, g = d[1], d[11]
    x = np.zeros(12)
    x[2] = w.SRB_COM_HEIGHT
    u = np.array([0.0, 0.0, 0.5 * m * g, 0.0, 0.0, 0.5 * m * g])
    f, _, _ = models.srb_fc(x[None], u[None], d)
    assert np.max(np.abs(f)) < 1e-12


def test_srb_torque_free_body_follows_eulers_equations():
    """No contact forces: free fall (v_dot = -g e_z) and Euler's equations of a
    rigid body with principal moments (Ixx, Iyy, Izz), written out per axis."""
    d = _srb_dyn()
    Ix, Iy, Iz, g = d[2], d[3], d[4], d[11]
    wx, wy, wz = 0.7, -1.3, 2.1
    x = np.zeros(12)
    x[6:9] = [0.2, -0.1, 0.4]
    x[9:12] = [wx, wy, wz]
    f, _, _ = models.srb_fc(x[None], np.zeros((1, 6)), d)
    assert np.allclose(f[0, 0:3], [0.2, -0.1, 0.4], atol=0, rtol=1e-15)
    assert np.allclose(f[0, 6:9], [0.0, 0.0, -g], atol=1e-15)
    expect = [(Iy - Iz) / Ix * wy * wz, (Iz - Ix) / Iy * wz * wx, (Ix - Iy) / Iz * wx * wy]
    assert np.allclose(f[0, 9:12], expect, rtol=1e-13, atol=1e-15)


def test_srb_euler_angle_rates():
    """ZYX Euler rates from body rates: identity when level; at zero roll
    theta_dot = (wx + tan(pitch) wz, wy, wz / cos(pitch)); at zero pitch a
    rotation of (wy, wz) by the roll angle."""
    d = _srb_dyn()
    om = np.array([0.3, -0.5, 0.9])
    for ang, expect in (((0.0, 0.0, 0.4), om),
                        ((0.0, 0.3, 0.0), [om[0] + np.tan(0.3) * om[2], om[1], om[2] / np.cos(0.3)]),
                        ((0.4, 0.0, 0.0), [om[0], np.cos(0.4) * om[1] - np.sin(0.4) * om[2],
                                           np.sin(0.4) * om[1] + np.cos(0.4) * om[2]])):
        x = np.zeros(12)
        x[3:6] = ang
        x[9:12] = om
        f, _, _ = models.srb_fc(x[None], np.zeros((1, 6)), d)
        assert np.allclose(f[0, 3:6], expect, rtol=1e-14, atol=1e-15), ang


def test_srb_foot_force_gives_r_cross_f():
    """One horizontal force on the left foot: acceleration f / m and angular
    acceleration (r_L x f) / I, the cross product written out."""
    d = _srb_dyn()
    m, Ix, Iy, Iz = d[1], d[2], d[3], d[4]
    rx, ry, rz = d[5], d[6], d[7]
    F = np.array([3.0, -2.0, 0.0])
    u = np.concatenate([F, np.zeros(3)])
    f, _, _ = models.srb_fc(np.zeros((1, 12)), u[None], d)
    tau = [ry * F[2] - rz * F[1], rz * F[0] - rx * F[2], rx * F[1] - ry * F[0]]
    assert np.allclose(f[0, 6:9], F / m + np.array([0, 0, -d[11]]), rtol=1e-14, atol=1e-15)
    assert np.allclose(f[0, 9:12], np.array(tau) / [Ix, Iy, Iz], rtol=1e-14, atol=1e-15)


def test_srb_rk4_is_exact_in_free_fall_and_constant_yaw_rate():
    """RK4 integrates polynomials of degree <= 4 exactly: a ballistic CoM
    (p + v dt - g dt^2 / 2 e_z) and a constant yaw rate at zero roll and pitch."""
    d = _srb_dyn()
    dt, g = d[0], d[11]
    x = np.zeros(12)
    x[0:3] = [0.1, 0.2, 0.7]
    x[5] = 0.3
    x[6:9] = [1.0, -0.5, 2.0]
    x[11] = 0.8
    phi, _, _ = models.rk4(models.srb_fc, x[None], np.zeros((1, 6)), d)
    p = x[0:3] + x[6:9] * dt + 0.5 * np.array([0, 0, -g]) * dt**2
    assert np.allclose(phi[0, 0:3], p, rtol=1e-14, atol=1e-15)
    assert np.allclose(phi[0, 6:9], x[6:9] + np.array([0, 0, -g]) * dt, rtol=1e-14, atol=1e-15)
    assert np.isclose(phi[0, 5], 0.3 + 0.8 * dt, rtol=1e-14)
    assert np.allclose(phi[0, 9:12], x[9:12], atol=1e-15)
