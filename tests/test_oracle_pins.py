"""Fixed-count pins of the oracle parts whose plausible mistakes survive the
converged-solution pins: the rho rule (Eq. rho:update) and the over-relaxation
of Algorithm 3 after one iteration, the line search of Appendix D on a worked
example, and the continuous-time models against closed-form motions.

Every expected number below is derived by hand in the docstring of its test
(a scalar QP, a one-interval double integrator, textbook rigid-body motions);
none is produced by running the oracle.
"""
import dataclasses
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as w
from oracle import admm as oadmm
from oracle import models as om
from oracle import sqp as osqp


# ---------------------------------------------------------------------------
# Algorithm 3: one over-relaxed iteration and one rho update on a scalar QP
# ---------------------------------------------------------------------------
def _scalar_qp(hi):
    """min 1/2 p x^2 + q x  s.t.  x = c (one equality row),  -10 <= x <= hi,
    with p = 2, q = 0, c = 1."""
    one = sp.csr_matrix(np.ones((1, 1)))
    return dict(P=sp.csr_matrix(np.array([[2.0]])), q=np.zeros(1), C=one, c=np.ones(1), G=one,
                lo=np.array([-10.0]), hi=np.array([hi]), gamma2=np.array([np.inf]), gamma1=np.zeros(1))


def _opts(**kw):
    return dataclasses.replace(w.Options(), **kw)


# Hand derivation (sigma = 1e-6, rho_bar = 1e-3: rho_f = 1, rho_g = 1e-3, alpha = 1.6,
# start x = z_g = y_f = y_g = 0):
#   S = p + sigma + rho_f + rho_g = 3.001001,  eta = -q + rho_f c = 1,  x~ = 1 / 3.001001
#   x^1 = alpha x~ = 1.6 / 3.001001 = 0.533155437135809          (over-relaxed primal)
#   z^_f = alpha x~ + (1 - alpha) c,  z^_g = alpha x~
#   y_f^1 = rho_f (z^_f - c) = 1.6 (x~ - 1) = -1.066844562864191
#   hi = 10:  z_g^1 = x^1, y_g^1 = 0
#   hi = 0.4: z_g^1 = 0.4, y_g^1 = rho_g (x^1 - 0.4) = 1.3315543713580903e-4
X1 = 1.6 / 3.001001
YF1 = 1.6 * (1.0 / 3.001001 - 1.0)


@pytest.mark.parametrize("hi,zg1,yg1", [(10.0, X1, 0.0), (0.4, 0.4, 1e-3 * (X1 - 0.4))], ids=["inactive", "active"])
def test_one_over_relaxed_iteration_by_hand(hi, zg1, yg1):
    r = oadmm.admm(_scalar_qp(hi), _opts(max_admm=1, k_rho_iter=10 ** 6, alpha=1.6), np.zeros(1), np.zeros(1),
                   np.zeros(1), np.zeros(1), 1e-3)
    assert r["x"][0] == pytest.approx(X1, rel=1e-12)
    assert r["yf"][0] == pytest.approx(YF1, rel=1e-12)
    assert r["zg"][0] == pytest.approx(zg1, rel=1e-12)
    assert r["yg"][0] == pytest.approx(yg1, rel=1e-9, abs=1e-18)


# The residuals after that iteration (hi = 10), Eq. admm:residuals:
#   r_prim = |x^1 - c| = 1 - 1.6/3.001001 = 0.46684456286419096
#   r_dual = |p x^1 + q + y_f^1 + y_g^1| = 0.0016016 / 3.001001 = 5.336885925729449e-4
#   prim normaliser max(|x^1|, |c|, |z_g|) = 1,  dual normaliser max(|p x^1|, |y_f^1|, |q|) = 3.2016016/3.001001
#   ratio = (0.46684456/1) / (5.3368859e-4 / 1.06684456) = 933.2232139
#   rho_new = 1e-3 sqrt(933.2232139) = 0.0305487023279531  (changes by 30.5 > 5: accepted)
# hi = 0.4: r_dual = |p x^1 + y_f^1 + y_g^1| = 4.0053315543713583e-4, dual normaliser
#   max(1.06631087, |y_f^1 + y_g^1| = 1.0667114074270552), ratio 1243.313852904468,
#   rho_new = 0.03526065587740064.
@pytest.mark.parametrize("hi,rho_new", [(10.0, 0.0305487023279531), (0.4, 0.03526065587740064)],
                         ids=["inactive", "active"])
def test_rho_update_by_hand(hi, rho_new):
    r = oadmm.admm(_scalar_qp(hi), _opts(max_admm=2, k_rho_iter=1, alpha=1.6), np.zeros(1), np.zeros(1),
                   np.zeros(1), np.zeros(1), 1e-3)
    assert len(r["rho_events"]) == 1
    k, rho = r["rho_events"][0]
    assert k == 1 and rho == pytest.approx(rho_new, rel=1e-10)


def test_rho_update_not_taken_below_the_ratio_threshold():
    """Same iteration with k_rho_ratio = 40 > 30.5: the candidate is not accepted."""
    r = oadmm.admm(_scalar_qp(10.0), _opts(max_admm=2, k_rho_iter=1, k_rho_ratio=40.0), np.zeros(1),
                   np.zeros(1), np.zeros(1), np.zeros(1), 1e-3)
    assert r["rho_events"] == [] and r["rho_bar"] == 1e-3


def test_rho_update_clipped_to_its_range():
    """rho_max = 0.01 < 0.0305: the candidate is clipped to 0.01 (ratio 10 > 5, accepted)."""
    r = oadmm.admm(_scalar_qp(10.0), _opts(max_admm=2, k_rho_iter=1, rho_max=0.01), np.zeros(1),
                   np.zeros(1), np.zeros(1), np.zeros(1), 1e-3)
    assert r["rho_events"] == [(1, 0.01)]


# ---------------------------------------------------------------------------
# Appendix D: a worked line search
# ---------------------------------------------------------------------------
def _di_one_interval():
    """Double integrator, N = 1, dt = 1 (A = [[I, I], [0, I]], B = [[I/2], [I]]),
    cost 1/2 (p_x,1 - 1)^2 only (Q = diag(1,0,0,0) on stage 1), no bounds."""
    pb = w.double_integrator(B=1, N=1)
    inst = pb.instance(0)
    inst["dyn"] = np.array([1.0])
    inst["x0"] = np.zeros(4)
    inst["Qd"] = np.array([[0.0, 0, 0, 0], [1.0, 0, 0, 0]])
    inst["Rd"] = np.zeros((2, 2))
    inst["Wd"] = np.zeros(2)
    inst["ref"] = np.zeros((2, 6))
    inst["ref"][1, 0] = 1.0
    inst["lin"] = np.zeros((2, 6))
    inst["lo"] = np.full((2, 4), -np.inf)
    inst["hi"] = np.full((2, 4), np.inf)
    return inst


def test_linesearch_worked_example():
    """Point z: x_0 = 0, u_0 = 0, x_1 = (0, 0.5, 0, 0) (dynamics residual f = (0, -0.5, 0, 0),
    V = 0.5).  Direction: u_0 = (8, 0), x_1 = B u_0 + (0, -0.5, 0, 0) = (4, -0.5, 8, 0).
    Along the line: p_x,1 = 4a, V(a) = 0.5 (1 - a), cost 1/2 (4a - 1)^2.
      grad l' d = (0 - 1) * 4 = -4;  mu = max(-4 / (0.5 * 0.5), ||y*|| + 1e-4) = 3.0001 (||y*|| = 3)
      phi(0) = 0.5 + 3.0001 * 0.5 = 2.00005;  D = -4 - 3.0001 * 0.5 = -5.50005
      phi(1) = 4.5,  phi(1/2) = 0.5 + 0.750025 = 1.250025,  phi(1/4) = 0 + 3.0001 * 0.375 = 1.1250375
      Armijo phi(a) <= 2.00005 + 0.4 a D:  a = 1: 4.5 > -0.20002;  a = 1/2: 1.250025 > 0.90004;
      a = 1/4: 1.1250375 <= 1.45005  ->  a = 1/4."""
    inst = _di_one_interval()
    z = np.zeros((2, 6))
    z[1, 1] = 0.5
    dz = np.zeros((2, 6))
    dz[0, 4] = 8.0
    dz[1, :4] = [4.0, -0.5, 8.0, 0.0]
    xi = np.zeros((2, 4))
    opts = _opts(n_ls=8, ls_eta=0.4, eps_c=1e-5)
    a, info = osqp.linesearch(inst, opts, z, xi, dz, np.zeros_like(xi), 3.0)
    assert a == 0.25
    assert info["mu"] == pytest.approx(3.0001, rel=1e-12)
    assert info["phi0"] == pytest.approx(2.00005, rel=1e-12)
    assert info["D"] == pytest.approx(-5.50005, rel=1e-12)
    assert info["phis"][:3] == pytest.approx([4.5, 1.250025, 1.1250375], rel=1e-12)


def test_linesearch_falls_back_to_least_merit():
    """An ascent direction (d = -u_0 of the example, no infeasibility): no candidate
    satisfies Armijo and the finite candidate of least merit is taken.  From
    z = 0 with V = 0: phi(a) = 1/2 (-4a - 1)^2 grows with a, so a = 2^-7."""
    inst = _di_one_interval()
    dz = np.zeros((2, 6))
    dz[0, 4] = -8.0
    dz[1, :4] = [-4.0, 0.0, -8.0, 0.0]
    xi = np.zeros((2, 4))
    a, info = osqp.linesearch(inst, _opts(n_ls=8), np.zeros((2, 6)), xi, dz, np.zeros_like(xi), 0.0)
    assert a == 2.0 ** -7
    assert info["phis"][-1] == pytest.approx(0.5 * (4 * 2.0 ** -7 + 1) ** 2, rel=1e-12)


# ---------------------------------------------------------------------------
# continuous-time models against closed-form motions
# ---------------------------------------------------------------------------
def _straight_track(heading=0.3, length=200.0, ds=w.TRACK_DS):
    """Table of a straight centreline through the origin with the given heading."""
    s = np.arange(0.0, length + ds / 2, ds)
    return np.stack([s * math.cos(heading), s * math.sin(heading), np.full_like(s, heading), np.zeros_like(s)], 1)


def _bicycle_dyn(L=2.7):
    return np.array([0.05, L, w.TRACK_DS, 400.0])


def test_bicycle_straight_line_at_zero_steering():
    """delta = 0: the car moves along its heading at speed v, heading constant;
    on a straight track of the same heading ds/dt = v, at a heading offset
    dpsi: ds/dt = v cos(dpsi)."""
    tab = _straight_track(0.3)
    x = np.array([[1.0, 2.0, 0.3, 7.0, 0.0, 10.0], [1.0, 2.0, 0.5, 7.0, 0.0, 10.0]])
    u = np.array([[0.7, -0.2], [0.7, -0.2]])
    f, _, _ = om.bicycle_fc(x, u, _bicycle_dyn(), tab)
    assert f[0] == pytest.approx([7 * math.cos(0.3), 7 * math.sin(0.3), 0.0, 0.7, -0.2, 7.0], abs=1e-12)
    assert f[1] == pytest.approx([7 * math.cos(0.5), 7 * math.sin(0.5), 0.0, 0.7, -0.2, 7 * math.cos(0.2)],
                                 abs=1e-12)


def test_bicycle_circle_at_constant_steering():
    """Constant steering delta and speed v: a circle of radius R = L / tan(delta)
    at yaw rate v tan(delta) / L.  The exact motion p(t) = c + R (sin psi(t),
    -cos psi(t)), psi(t) = psi_0 + v tan(delta) t / L has dp/dt = v (cos psi, sin psi),
    which the model must return at every point of the circle."""
    L, v, dl = 2.7, 9.0, 0.25
    R = L / math.tan(dl)
    om_ = v * math.tan(dl) / L
    tab = _straight_track(0.0)
    for t in (0.0, 0.7, 2.3):
        psi = 0.4 + om_ * t
        p = np.array([3.0 + R * math.sin(psi), -1.0 - R * math.cos(psi)])
        x = np.array([[p[0], p[1], psi, v, dl, 5.0]])
        f, _, _ = om.bicycle_fc(x, np.zeros((1, 2)), _bicycle_dyn(L), tab)
        dp = np.array([R * math.cos(psi) * om_, R * math.sin(psi) * om_])
        assert f[0, :3] == pytest.approx([dp[0], dp[1], om_], rel=1e-12)
        assert math.hypot(f[0, 0], f[0, 1]) == pytest.approx(om_ * R, rel=1e-12)   # = v


def test_quadrotor_hover_and_rigid_body_motion():
    """Planar quadrotor (m, I, arm, g): at rest with thrusts m g / 2 each f_c = 0;
    with no thrust, free fall (z'' = -g); a tilt theta with total thrust T gives
    x'' = -T sin(theta) / m, z'' = T cos(theta) / m - g; a thrust difference gives
    omega' = (T2 - T1) arm / I."""
    dyn = np.array([0.05, 1.0, 0.01, 0.1, 9.81])
    m, I, arm, g = 1.0, 0.01, 0.1, 9.81
    x = np.array([[0.3, -2.0, 0.0, 0.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 1.5, -0.5, 0.2],
                  [0.0, 0.0, math.pi / 6, 0.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 0.0, 0.0, 0.0]])
    u = np.array([[m * g / 2, m * g / 2], [0.0, 0.0], [6.0, 6.0], [4.0, 5.0]])
    f, _, _ = om.quad_fc(x, u, dyn)
    assert f[0] == pytest.approx(np.zeros(6), abs=1e-12)
    assert f[1] == pytest.approx([1.5, -0.5, 0.2, 0.0, -g, 0.0], abs=1e-12)
    assert f[2] == pytest.approx([0, 0, 0, -12.0 * 0.5 / m, 12.0 * math.cos(math.pi / 6) / m - g, 0], abs=1e-12)
    assert f[3] == pytest.approx([0, 0, 0, 0, 9.0 / m - g, (5.0 - 4.0) * arm / I], abs=1e-12)


def test_quadrotor_rk4_is_exact_for_ballistic_flight():
    """With zero thrust and zero angular rate the motion is a parabola, which
    RK4 integrates exactly: z(dt) = z + v_z dt - g dt^2 / 2, v_z(dt) = v_z - g dt."""
    dt, g = 0.05, 9.81
    dyn = np.array([dt, 1.0, 0.01, 0.1, g])
    x = np.array([[0.3, 1.0, 0.2, 2.0, 1.5, 0.0]])
    phi, _, _ = om.quad_rk4(x, np.zeros((1, 2)), dyn)
    assert phi[0] == pytest.approx([0.3 + 2.0 * dt, 1.0 + 1.5 * dt - 0.5 * g * dt * dt, 0.2, 2.0, 1.5 - g * dt, 0.0],
                                   abs=1e-13)


def test_midpoint_rule_is_exact_for_uniform_motion():
    """The implicit midpoint constraint x_{t+1} = x_t + dt f_c((x_t + x_{t+1}) / 2, u_t)
    holds exactly for a straight line at constant speed on a straight track
    aligned with it (every derivative of f_c along that motion vanishes)."""
    tab = _straight_track(0.3)
    dyn = _bicycle_dyn()
    dt, v = dyn[0], 8.0
    N = 4
    z = np.zeros((N + 1, 8))
    for t in range(N + 1):
        s = 5.0 + v * dt * t
        z[t, :6] = [s * math.cos(0.3), s * math.sin(0.3), 0.3, v, 0.0, s]
    inst = dict(model=w.MODEL_BICYCLE, nx=6, nu=2, dyn=dyn, track=tab)
    f, _, _ = om.dynamics(inst, z)
    assert np.max(np.abs(f)) < 1e-12
