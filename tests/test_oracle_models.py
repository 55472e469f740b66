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
