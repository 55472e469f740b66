"""Seeded synthetic problem generators for the batched OCP solver.

This module only draws numbers: initial states, cost weights, references,
bounds, slack weights, dynamics parameters and track tables.  It holds none of
the solver's arithmetic (no linearisation, no QP assembly, no ADMM), so both
the FP64 oracle and the CUDA path can consume its output without sharing any
method code.

Problem family (the OCP of Section II-A / Appendix A of the paper):

    min  sum_t l_t(z_t, z_{t+1}) + l_N(z_N) + slack penalties
    s.t. x_0 = x_init,  f_t(z_t, z_{t+1}) = 0,  lo_t <= g_t(z_t) + xi_t <= hi_t

with z_t = (x_t, u_t) stacked per stage, t = 0..N.  The stage cost is
diagonal-quadratic with an optional control-rate term (the racing cost of
Eq. (cost) in Section V):

    l_t = 1/2 (x_t-xr_t)' Q_t (x_t-xr_t) + 1/2 (u_t-ur_t)' R_t (u_t-ur_t)
          + 1/2 (u_t-u_{t+1})' W (u_t-u_{t+1}) + lin_t' z_t
    l_N = 1/2 (x_N-xr_N)' Q_N (x_N-xr_N) + 1/2 (u_N-ur_N)' R_N (u_N-ur_N)
          + lin_N' z_N

Layout (padded batch, float64 here; the CUDA path casts to float32):
    N      [B]               horizon of each instance (stages 0..N)
    model  [B]               MODEL_* id
    x0     [B][nx]
    Qd     [B][Nm+1][nx]     diagonal state weights (row N = terminal)
    Rd     [B][Nm+1][nu]
    Wd     [B][nu]           control-rate weights
    ref    [B][Nm+1][n]      (x_ref, u_ref)
    lin    [B][Nm+1][n]      linear cost term
    lo, hi [B][Nm+1][ng]     bounds on g_t (+-inf = no bound)
    gamma2 [B][ng]           L2 slack weight per constraint row; inf = hard row
    gamma1 [B][ng]           L1 slack weight per constraint row
    dyn    [B][n_dyn]        model parameters (see MODEL_* below)
    track  [B][n_track+1][4] centreline table (x_c, y_c, psi_c, kappa) or None

An instance whose model has smaller (nx, nu, ng) than the layout uses the
leading entries of each stage vector: z[t][:nx_i] is the state and
z[t][nx_i:nx_i+nu_i] the control; the rest is padding.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MODEL_DI = 0        # 2-D double integrator, ZOH.          dyn = [dt]
MODEL_LINEAR = 1    # x+ = A x + B u + b (explicit).       dyn = [A (nx*nx), B (nx*nu), b (nx, optional)] row-major
MODEL_BICYCLE = 2   # kinematic bicycle, implicit midpoint. dyn = [dt, wheelbase, ds, n_track]
MODEL_QUAD = 3      # planar quadrotor, explicit RK4.       dyn = [dt, mass, inertia, arm, gravity]
MODEL_BICYCLE_TRAP = 4    # kinematic bicycle, trapezoidal rule (implicit).        dyn as MODEL_BICYCLE
MODEL_BICYCLE_NEWTON = 5  # kinematic bicycle, explicit map x+ = Phi(x, u) defined by 3 Newton steps
                          # on the implicit midpoint rule, Jacobians by the implicit function theorem
MODEL_SRB = 6       # single-rigid-body humanoid, explicit RK4. dyn = [dt, mass, Ixx, Iyy, Izz, r_L (3), r_R (3), gravity]

MODEL_NAMES = {MODEL_DI: "double_integrator", MODEL_LINEAR: "linear",
               MODEL_BICYCLE: "bicycle", MODEL_QUAD: "planar_quadrotor",
               MODEL_BICYCLE_TRAP: "bicycle_trapezoidal", MODEL_BICYCLE_NEWTON: "bicycle_newton_map",
               MODEL_SRB: "srb_humanoid"}
BICYCLES = (MODEL_BICYCLE, MODEL_BICYCLE_TRAP, MODEL_BICYCLE_NEWTON)
INTEGRATORS = {"midpoint": MODEL_BICYCLE, "trapezoidal": MODEL_BICYCLE_TRAP, "newton_map": MODEL_BICYCLE_NEWTON}

# fixed (nx, nu, ng) of the nonlinear / fixed-size models
MODEL_DIMS = {MODEL_DI: (4, 2, 4), MODEL_BICYCLE: (6, 2, 5), MODEL_QUAD: (6, 2, 2),
              MODEL_BICYCLE_TRAP: (6, 2, 5), MODEL_BICYCLE_NEWTON: (6, 2, 5), MODEL_SRB: (12, 6, 6)}

# rows of g that bound one stage variable directly (its index), -1 for other rows;
# the linear and SRB models bound their controls (index nx + r) and are not listed
SELECTOR_ROWS = {MODEL_DI: (4, 5, 2, 3), MODEL_QUAD: (6, 7), MODEL_BICYCLE: (6, 7, 3, 4, -1),
                 MODEL_BICYCLE_TRAP: (6, 7, 3, 4, -1), MODEL_BICYCLE_NEWTON: (6, 7, 3, 4, -1)}

INF = np.inf


def model_dims(model: int, nx: int, nu: int, ng: int):
    """(nx, nu, ng) of one instance; the linear model uses the layout dims."""
    if model == MODEL_LINEAR:
        return nx, nu, ng
    return MODEL_DIMS[model]


@dataclasses.dataclass
class Options:
    """Solver options (the defaults follow Sections III-B/III-C of the paper)."""
    sigma: float = 1e-6
    rho0: float = 0.1
    rho_min: float = 1e-6
    rho_max: float = 1e6
    alpha: float = 1.6          # over-relaxation (value not given in the paper)
    eps_abs: float = 1e-5
    eps_rel: float = 1e-5
    eps_c: float = 1e-5
    eps_g: float = 1e-4
    ls_eta: float = 0.4
    k_rho_iter: int = 25
    k_rho_ratio: float = 5.0
    max_sqp: int = 1
    max_admm: int = 200
    n_ls: int = 8
    newton_steps: int = 3
    early_exit: int = 0
    check_every: int = 25
    bwd_rho: float = 1e4
    bwd_sigma: float = 1e-6
    bwd_iters: int = 30
    bwd_gamma: float = 1e4      # penalty weight of hard active rows in the reduced adjoint QP


@dataclasses.dataclass
class ProblemBatch:
    nx: int
    nu: int
    ng: int
    N_max: int
    N: np.ndarray
    model: np.ndarray
    x0: np.ndarray
    Qd: np.ndarray
    Rd: np.ndarray
    Wd: np.ndarray
    ref: np.ndarray
    lin: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    gamma2: np.ndarray
    gamma1: np.ndarray
    dyn: np.ndarray
    track: np.ndarray | None
    opts: Options
    name: str = ""
    z_init: np.ndarray | None = None   # [B][Nm+1][n] initial primal guess (warm start), or None
    scale: np.ndarray | None = None    # [B][n] characteristic magnitude of each state / control, or None
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def B(self) -> int:
        return int(self.N.shape[0])

    @property
    def n(self) -> int:
        return self.nx + self.nu

    @property
    def n_dyn(self) -> int:
        return int(self.dyn.shape[1])

    @property
    def n_track(self) -> int:
        return 0 if self.track is None else int(self.track.shape[1]) - 1

    def dims_of(self, i: int):
        return model_dims(int(self.model[i]), self.nx, self.nu, self.ng)

    def instance(self, i: int) -> dict:
        """One instance, unpadded (stage arrays cut to N_i+1 and model dims)."""
        nx, nu, ng = self.dims_of(i)
        Ni = int(self.N[i])
        T = Ni + 1
        # padded layout keeps the state in [:nx_i] and the control in [nx_i:nx_i+nu]
        ref = self.ref[i, :T, :nx + nu].copy()
        lin = self.lin[i, :T, :nx + nu].copy()
        tr = None
        if self.track is not None and int(self.model[i]) in BICYCLES:
            nt = int(round(self.dyn[i, 3]))
            tr = self.track[i, :nt + 1].copy()
        z0 = None if self.z_init is None else self.z_init[i, :T, :nx + nu].copy()
        sc = None if self.scale is None else self.scale[i, :nx + nu].copy()
        return dict(model=int(self.model[i]), N=Ni, nx=nx, nu=nu, ng=ng, z_init=z0, scale=sc,
                    x0=self.x0[i, :nx].copy(), Qd=self.Qd[i, :T, :nx].copy(),
                    Rd=self.Rd[i, :T, :nu].copy(), Wd=self.Wd[i, :nu].copy(),
                    ref=ref, lin=lin, lo=self.lo[i, :T, :ng].copy(),
                    hi=self.hi[i, :T, :ng].copy(), gamma2=self.gamma2[i, :ng].copy(),
                    gamma1=self.gamma1[i, :ng].copy(), dyn=self.dyn[i].copy(), track=tr)

    def subset(self, idx) -> "ProblemBatch":
        idx = np.asarray(idx)
        def s(a):
            return None if a is None else a[idx].copy()
        return dataclasses.replace(
            self, N=s(self.N), model=s(self.model), x0=s(self.x0), Qd=s(self.Qd),
            Rd=s(self.Rd), Wd=s(self.Wd), ref=s(self.ref), lin=s(self.lin), lo=s(self.lo),
            hi=s(self.hi), gamma2=s(self.gamma2), gamma1=s(self.gamma1), dyn=s(self.dyn),
            track=s(self.track), z_init=s(self.z_init), scale=s(self.scale), extra=dict(self.extra))


def magnitude_scales(pb: "ProblemBatch", floor: float = 1.0) -> np.ndarray:
    """Characteristic magnitude of every state and control of each instance:
    the largest |value| the component takes in the initial guess (z_init, else
    x0 for the states), or the largest finite bound of a row that bounds the
    component alone, floored at `floor`.  Input data for the solver's optional
    normalisation of states and controls (a user's choice of units, like the
    bounds themselves); [B][n]."""
    B, n = pb.B, pb.n
    out = np.full((B, n), float(floor))
    for i in range(B):
        nx, nu, ng = pb.dims_of(i)
        T = int(pb.N[i]) + 1
        mag = np.zeros(n)
        if pb.z_init is not None:
            mag[:nx + nu] = np.max(np.abs(pb.z_init[i, :T, :nx + nu]), axis=0)
        else:
            mag[:nx] = np.abs(pb.x0[i, :nx])
        for r, j in enumerate(SELECTOR_ROWS.get(int(pb.model[i]), ())):
            if j < 0 or r >= ng:
                continue
            b = np.concatenate([pb.lo[i, :T, r], pb.hi[i, :T, r]])
            b = np.abs(b[np.isfinite(b)])
            if b.size:
                mag[j] = max(mag[j], float(np.max(b)))
        out[i] = np.maximum(mag, floor)
    return out


def _empty(B, nx, nu, ng, N_max, n_dyn, n_track):
    n = nx + nu
    T = N_max + 1
    return dict(
        x0=np.zeros((B, nx)), Qd=np.zeros((B, T, nx)), Rd=np.zeros((B, T, nu)),
        Wd=np.zeros((B, nu)), ref=np.zeros((B, T, n)), lin=np.zeros((B, T, n)),
        lo=np.full((B, T, ng), -INF), hi=np.full((B, T, ng), INF),
        gamma2=np.full((B, ng), INF), gamma1=np.zeros((B, ng)),
        dyn=np.zeros((B, n_dyn)),
        track=None if n_track == 0 else np.zeros((B, n_track + 1, 4)))


# ----------------------------------------------------------------------------
# tracks (geometry only)
# ----------------------------------------------------------------------------
TRACK_DS = 0.5      # centreline table spacing [m]


def open_spline_track(rng, length=400.0, knot_every=10.0, kappa_max=0.2, ds=TRACK_DS):
    """Centreline whose curvature is a C2 cubic spline through knots drawn from
    U[-kappa_max, kappa_max] every `knot_every` metres; heading and position are
    integrated from the curvature on a fine grid and tabulated every `ds`."""
    from scipy.interpolate import CubicSpline
    n_knots = int(math.ceil(length / knot_every)) + 2
    sk = np.arange(n_knots) * knot_every
    kk = rng.uniform(-kappa_max, kappa_max, size=n_knots)
    spline = CubicSpline(sk, kk, bc_type="natural")
    fine = 0.01
    sf = np.arange(0.0, length + fine / 2, fine)
    kf = spline(sf)
    psi = np.concatenate([[0.0], np.cumsum(0.5 * (kf[1:] + kf[:-1]) * fine)])
    psi += rng.uniform(-math.pi, math.pi)
    c, s = np.cos(psi), np.sin(psi)
    x = np.concatenate([[0.0], np.cumsum(0.5 * (c[1:] + c[:-1]) * fine)])
    y = np.concatenate([[0.0], np.cumsum(0.5 * (s[1:] + s[:-1]) * fine)])
    step = int(round(ds / fine))
    sel = np.arange(0, len(sf), step)
    tab = np.stack([x[sel], y[sel], psi[sel], kf[sel]], axis=1)
    return tab  # n_track+1 rows, n_track = length/ds


def closed_track(rng, length=2000.0, harmonics=12, ds=TRACK_DS, kappa_max=0.2):
    """Closed, counter-clockwise centreline r(phi) = R0 (1 + sum a_k cos(k phi + p_k)),
    rescaled to the requested length and tabulated every `ds` by arc length.
    The last row repeats the first point with heading + 2*pi (periodic table)."""
    M = 200000
    phi = np.linspace(0.0, 2 * math.pi, M, endpoint=False)
    for _ in range(50):
        a = rng.normal(0, 1, harmonics) / (np.arange(2, harmonics + 2) ** 2) * 0.25
        p = rng.uniform(0, 2 * math.pi, harmonics)
        r = np.ones_like(phi)
        for k in range(harmonics):
            r += a[k] * np.cos((k + 2) * phi + p[k])
        if r.min() < 0.3:
            continue
        x, y = r * np.cos(phi), r * np.sin(phi)
        dx = np.roll(x, -1) - x
        dy = np.roll(y, -1) - y
        seg = np.hypot(dx, dy)
        L = seg.sum()
        scale = length / L
        x, y, seg = x * scale, y * scale, seg * scale
        s = np.concatenate([[0.0], np.cumsum(seg)[:-1]])
        psi = np.unwrap(np.arctan2(dy, dx))
        # curvature by finite differences of the heading along arc length
        dpsi = np.diff(np.concatenate([psi, [psi[0] + 2 * math.pi]]))
        kap = dpsi / seg
        if np.max(np.abs(kap)) > kappa_max:
            continue
        n_track = int(round(length / ds))
        sq = np.arange(n_track) * ds
        xs = np.interp(sq, s, x, period=length)
        ys = np.interp(sq, s, y, period=length)
        psi_s = np.interp(sq, np.concatenate([s, [length]]), np.concatenate([psi, [psi[0] + 2 * math.pi]]))
        k_s = np.interp(sq, s, kap, period=length)
        tab = np.stack([xs, ys, psi_s, k_s], axis=1)
        last = np.array([[xs[0], ys[0], psi_s[0] + 2 * math.pi, k_s[0]]])
        return np.concatenate([tab, last], axis=0)
    raise RuntimeError("closed_track: could not draw a track within the curvature bound")


def centreline_guess(tab, N, dt, v0, wheelbase, ds=TRACK_DS):
    """Initial guess that follows the centreline at constant speed v0: stage t sits at
    arc length s_t = v0 t dt on the centreline with the centreline heading, the
    steering angle atan(wheelbase kappa(s_t)) and zero acceleration (geometry of
    the table only, linear interpolation; not dynamically exact)."""
    nt = tab.shape[0] - 1
    L = nt * ds
    s = v0 * dt * np.arange(N + 1)
    sm = np.mod(s, L)
    grid = np.arange(nt + 1) * ds
    xc = np.interp(sm, grid, tab[:, 0])
    yc = np.interp(sm, grid, tab[:, 1])
    psi = np.interp(sm, grid, tab[:, 2]) + 2 * np.pi * np.floor(s / L)
    kap = np.interp(sm, grid, tab[:, 3])
    dl = np.arctan(wheelbase * kap)
    z = np.zeros((N + 1, 8))
    z[:, 0], z[:, 1], z[:, 2], z[:, 3], z[:, 4], z[:, 5] = xc, yc, psi, v0, dl, s
    z[:-1, 7] = np.diff(dl) / dt
    return z


# ----------------------------------------------------------------------------
# per-model instance fillers
# ----------------------------------------------------------------------------
def _fill_di(rng, a, i, N, nx_l, nu_l, dt=0.05, x0=None):
    nx, nu = 4, 2
    q = rng.uniform(1.0, 10.0, size=nx)
    a["Qd"][i, :N, :nx] = q
    a["Qd"][i, N, :nx] = 10.0 * q
    a["Rd"][i, :N + 1, :nu] = 0.1
    a["x0"][i, :nx] = rng.normal(0, 1, nx) if x0 is None else x0
    # rows: u1, u2, vx, vy;  |u| <= 1 on t = 0..N, |v| <= 2 on t = 1..N
    a["lo"][i, :N + 1, 0:2] = -1.0
    a["hi"][i, :N + 1, 0:2] = 1.0
    a["lo"][i, 1:N + 1, 2:4] = -2.0
    a["hi"][i, 1:N + 1, 2:4] = 2.0
    a["dyn"][i, 0] = dt
    if "z_init" in a:
        a["z_init"][i, :N + 1, :nx] = a["x0"][i, :nx]


def _fill_bicycle(rng, a, i, N, track_tab, dt=0.05, wheelbase=2.7, v0=None,
                  gamma2=100.0, gamma1=10.0, w_progress=1.0):
    nx, nu = 6, 2
    # cost: steering-angle regularisation, control effort, control rate, progress
    a["Qd"][i, :N + 1, :nx] = np.array([0.0, 0.0, 0.0, 0.0, 0.1, 0.0])
    a["Rd"][i, :N + 1, :nu] = np.array([0.01, 0.1])
    a["Wd"][i, :nu] = np.array([0.1, 0.1])
    a["lin"][i, N, 5] = -w_progress                       # min-time: -w_s * s_N
    xc, yc, psic = track_tab[0, 0], track_tab[0, 1], track_tab[0, 2]
    v = rng.uniform(5.0, 15.0) if v0 is None else v0
    a["x0"][i, :nx] = np.array([xc, yc, psic, v, 0.0, 0.0])
    a["ref"][i, :N + 1, 3] = v                            # unused (zero weight) but recorded
    # rows: accel, steer-rate, speed, steering angle, lateral error e
    a["lo"][i, :N + 1, 0] = -4.0
    a["hi"][i, :N + 1, 0] = 4.0
    a["lo"][i, :N + 1, 1] = -1.0
    a["hi"][i, :N + 1, 1] = 1.0
    a["lo"][i, 1:N + 1, 2] = 0.0
    a["hi"][i, 1:N + 1, 2] = 30.0
    a["lo"][i, 1:N + 1, 3] = -0.6
    a["hi"][i, 1:N + 1, 3] = 0.6
    a["lo"][i, 1:N + 1, 4] = -4.0
    a["hi"][i, 1:N + 1, 4] = 4.0
    a["gamma2"][i, :] = INF
    a["gamma1"][i, :] = 0.0
    a["gamma2"][i, 4] = gamma2                            # track row is softened (L1 + L2)
    a["gamma1"][i, 4] = gamma1
    nt = track_tab.shape[0] - 1
    a["dyn"][i, 0:4] = np.array([dt, wheelbase, TRACK_DS, nt])
    a["track"][i, :nt + 1] = track_tab
    if "z_init" in a:
        a["z_init"][i, :N + 1, :8] = centreline_guess(track_tab, N, dt, v, wheelbase)


QUAD_MASS, QUAD_INERTIA, QUAD_ARM, GRAVITY = 1.0, 0.01, 0.1, 9.81


def _fill_quad(rng, a, i, N, dt=0.05):
    nx, nu = 6, 2
    hover = QUAD_MASS * GRAVITY / 2.0
    a["Qd"][i, :N + 1, :nx] = np.array([10.0, 10.0, 1.0, 1.0, 1.0, 0.1])
    a["Qd"][i, N, :nx] *= 10.0
    a["Rd"][i, :N + 1, :nu] = 0.1
    a["ref"][i, :N + 1, nx:nx + nu] = hover
    a["x0"][i, :nx] = rng.normal(0, 1, nx) * np.array([0.5, 0.5, 0.2, 0.5, 0.5, 0.5])
    a["lo"][i, :N + 1, 0:2] = 0.0
    a["hi"][i, :N + 1, 0:2] = 10.0
    a["dyn"][i, 0:5] = np.array([dt, QUAD_MASS, QUAD_INERTIA, QUAD_ARM, GRAVITY])
    if "z_init" in a:
        a["z_init"][i, :N + 1, :nx] = a["x0"][i, :nx]
        a["z_init"][i, :N + 1, nx:nx + nu] = hover


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------
def double_integrator(B=1, N=20, seed=1001, max_admm=200) -> ProblemBatch:
    """Linear 2-D double integrator (nx=4, nu=2), ZOH dt=0.05, horizon N.
    Q = diag(U[1,10]), R = 0.1 I, Q_N = 10 Q, x0 ~ N(0, I), |u| <= 1, |v| <= 2.
    One SQP step (the problem is already a QP), `max_admm` ADMM iterations."""
    rng = np.random.default_rng(seed)
    nx, nu, ng = 4, 2, 4
    a = _empty(B, nx, nu, ng, N, 1, 0)
    for i in range(B):
        _fill_di(np.random.default_rng([seed, i]), a, i, N, nx, nu)
    opts = Options(max_sqp=1, max_admm=max_admm, n_ls=1)
    return ProblemBatch(nx, nu, ng, N, np.full(B, N, np.int32), np.full(B, MODEL_DI, np.int32),
                        opts=opts, name=f"double_integrator_B{B}_N{N}", **a)


def racing(B=1024, N=50, seed=1002, max_sqp=10, max_admm=50, track_length=400.0,
           integrator="midpoint") -> ProblemBatch:
    """Kinematic-bicycle racing (nx=6: x, y, psi, v, delta, s; nu=2: accel,
    steer-rate), implicit midpoint dt=0.05, N=50, random curvature-spline
    centrelines (curvature knots every 10 m in U[-0.2, 0.2]), box bounds on the
    controls, speed and steering angle, the lateral track error softened by L1+L2 slacks,
    control-rate cost and a min-time (progress) terminal cost.  integrator:
    "midpoint" (the implicit midpoint constraint), "trapezoidal" (the trapezoidal
    constraint) or "newton_map" (the explicit map defined by 3 Newton steps on
    the midpoint rule)."""
    nx, nu, ng = 6, 2, 5
    nt = int(round(track_length / TRACK_DS))
    a = _empty(B, nx, nu, ng, N, 4, nt)
    a["z_init"] = np.zeros((B, N + 1, nx + nu))
    for i in range(B):
        r = np.random.default_rng([seed, i])
        tab = open_spline_track(r, length=track_length)
        _fill_bicycle(r, a, i, N, tab)
    opts = Options(max_sqp=max_sqp, max_admm=max_admm, n_ls=8)
    return ProblemBatch(nx, nu, ng, N, np.full(B, N, np.int32), np.full(B, INTEGRATORS[integrator], np.int32),
                        opts=opts, name=f"racing_B{B}_N{N}" + ("" if integrator == "midpoint" else "_" + integrator),
                        **a)


def mlp_init(rng, sizes=(16, 64, 64, 68)):
    """Random weights of the tanh cost MLP (context -> log cost weights)."""
    params = []
    for k in range(len(sizes) - 1):
        fan_in = sizes[k]
        scale = 1.0 / math.sqrt(fan_in) if k < len(sizes) - 2 else 0.3 / math.sqrt(fan_in)
        W = rng.normal(0, scale, size=(sizes[k + 1], sizes[k]))
        b = np.zeros(sizes[k + 1])
        params += [W, b]
    return params


def mlp_forward_np(params, ctx):
    """Plain numpy forward of the cost MLP (tanh hidden layers, linear output)."""
    h = ctx
    L = len(params) // 2
    for k in range(L):
        W, b = params[2 * k], params[2 * k + 1]
        h = h @ W.T + b
        if k < L - 1:
            h = np.tanh(h)
    return h


R_SCALE_TRACKING = 0.1


def tracking(B=512, nx=48, nu=20, N=32, seed=1003, max_admm=200, dt=0.05) -> ProblemBatch:
    """Differentiable tracking: random stable linear dynamics nx=48, nu=20, N=32,
    A = I + dt (S - 0.1 I) with S = (M - M')/sqrt(2), M_ij ~ N(0, 1/nx); B_ij ~ N(0, 1/nx).
    Reference: sinusoids with random frequency and phase; |u| <= 1.  Cost weights
    Q = exp(o[:nx]), R = 0.1 exp(o[nx:]) with o = MLP(context), context ~ N(0, I_16),
    MLP 16 -> 64 -> 64 -> nx+nu with tanh hidden layers."""
    rng = np.random.default_rng(seed)
    ng = nu
    n = nx + nu
    n_dyn = nx * nx + nx * nu
    a = _empty(B, nx, nu, ng, N, n_dyn, 0)
    mlp = mlp_init(rng, (16, 64, 64, n))
    ctx = rng.normal(0, 1, size=(B, 16))
    out = mlp_forward_np(mlp, ctx)
    Mmat = rng.normal(0, 1.0 / math.sqrt(nx), size=(nx, nx))
    S = (Mmat - Mmat.T) / math.sqrt(2.0)
    A = np.eye(nx) + dt * (S - 0.1 * np.eye(nx))
    Bm = rng.normal(0, 1.0 / math.sqrt(nx), size=(nx, nu))
    tgrid = np.arange(N + 1) * dt
    for i in range(B):
        r = np.random.default_rng([seed, i])
        a["Qd"][i, :, :] = np.exp(out[i, :nx])
        a["Rd"][i, :, :] = R_SCALE_TRACKING * np.exp(out[i, nx:])
        a["x0"][i] = r.normal(0, 1, nx)
        omega = r.uniform(0.5, 2.0)
        phase = r.uniform(0, 2 * math.pi, nx)
        a["ref"][i, :, :nx] = np.sin(omega * tgrid[:, None] + phase[None, :])
        a["lo"][i, :, :] = -1.0
        a["hi"][i, :, :] = 1.0
        a["dyn"][i, :nx * nx] = A.ravel()
        a["dyn"][i, nx * nx:] = Bm.ravel()
    opts = Options(max_sqp=1, max_admm=max_admm, n_ls=1)
    pb = ProblemBatch(nx, nu, ng, N, np.full(B, N, np.int32), np.full(B, MODEL_LINEAR, np.int32),
                      opts=opts, name=f"tracking_B{B}_nx{nx}_nu{nu}_N{N}", **a)
    pb.extra = dict(mlp=mlp, ctx=ctx, spectral_radius=float(np.max(np.abs(np.linalg.eigvals(A)))))
    return pb


def uneven(B=4096, N_lo=10, N_hi=200, seed=1004, max_sqp=10, max_admm=50) -> ProblemBatch:
    """Uneven batch: each instance draws its horizon from U{N_lo..N_hi} and its
    model from {double integrator, bicycle, planar quadrotor} with ratio 1:2:1."""
    rng = np.random.default_rng(seed)
    nx, nu, ng = 6, 2, 5
    Ns = rng.integers(N_lo, N_hi + 1, size=B).astype(np.int32)
    models = rng.choice([MODEL_DI, MODEL_BICYCLE, MODEL_BICYCLE, MODEL_QUAD], size=B).astype(np.int32)
    N_max = int(Ns.max())
    track_len = 400.0
    nt = int(round(track_len / TRACK_DS))
    a = _empty(B, nx, nu, ng, N_max, 5, nt)
    a["z_init"] = np.zeros((B, N_max + 1, nx + nu))
    for i in range(B):
        r = np.random.default_rng([seed, i])
        if models[i] == MODEL_DI:
            _fill_di(r, a, i, int(Ns[i]), nx, nu)
        elif models[i] == MODEL_BICYCLE:
            _fill_bicycle(r, a, i, int(Ns[i]), open_spline_track(r, length=track_len))
        else:
            _fill_quad(r, a, i, int(Ns[i]))
    opts = Options(max_sqp=max_sqp, max_admm=max_admm, n_ls=8)
    return ProblemBatch(nx, nu, ng, N_max, Ns, models, opts=opts,
                        name=f"uneven_B{B}_N{N_lo}-{N_hi}", **a)


def long_horizon(B=8, N=8192, seed=1005, max_sqp=5, max_admm=100, dt=0.01,
                 track_length=2000.0) -> ProblemBatch:
    """Kinematic-bicycle racing as `racing`, with N=8192 knots at dt=0.01 on a
    closed random track of 2 km."""
    nx, nu, ng = 6, 2, 5
    nt = int(round(track_length / TRACK_DS))
    a = _empty(B, nx, nu, ng, N, 4, nt)
    a["z_init"] = np.zeros((B, N + 1, nx + nu))
    for i in range(B):
        r = np.random.default_rng([seed, i])
        tab = closed_track(r, length=track_length)
        _fill_bicycle(r, a, i, N, tab, dt=dt)
    opts = Options(max_sqp=max_sqp, max_admm=max_admm, n_ls=8)
    return ProblemBatch(nx, nu, ng, N, np.full(B, N, np.int32), np.full(B, MODEL_BICYCLE, np.int32),
                        opts=opts, name=f"long_horizon_B{B}_N{N}", **a)


def stable_linear_system(rng, nx, nu, scale=0.1, lam_max=0.99, b_std=1e-2):
    """A = I + scale * dA with dA_ij ~ N(0, 1) and its eigenvalues scaled onto the
    disc |lambda| <= lam_max (A = V diag(lambda) V^-1 with each lambda that lies
    outside multiplied by lam_max / |lambda|; conjugate pairs stay conjugate, so A
    stays real); B_ij ~ N(0, 1); b ~ N(0, b_std^2 I)."""
    A = np.eye(nx) + scale * rng.normal(0, 1, size=(nx, nx))
    lam, V = np.linalg.eig(A)
    lam = lam * np.minimum(1.0, lam_max / np.maximum(np.abs(lam), 1e-300))
    A = np.real(V @ np.diag(lam) @ np.linalg.inv(V))
    B = rng.normal(0, 1, size=(nx, nu))
    b = rng.normal(0, b_std, size=nx)
    return A, B, b


def linear_rl(B=64, N=40, nx=8, nu=4, u_max=1.0, seed=1006, theta=None, tol=1e-5, max_admm=1000,
              max_sqp=10, rho_max=1.0) -> ProblemBatch:
    """The linear-system RL problem family: x+ = A x + B u + b (one system drawn
    per seed, see stable_linear_system), x0 ~ N(0, 25 I) per instance, stage
    cost x' Q x + ||u||^2 with Q = diag(theta) (written with the 1/2 of the
    cost convention: Qd = 2 theta, Rd = 2; theta = 1 unless given), the same
    cost at the terminal stage, control box |u|_inf <= u_max on every stage.
    The solver runs to the tolerance tol (early exit at eps_abs = eps_rel =
    eps_c = tol) with at most max_admm ADMM iterations per QP.  rho_bar is
    capped at rho_max = 1 (rho_f <= 1e3): with x0 ~ N(0, 25 I) and saturated
    controls the rho rule asks for rho_bar ~ 10, where S reaches a condition
    number near 1e5 and an FP32 solve no longer keeps the ADMM iteration
    stable (an FP64 run with S perturbed by one FP32 rounding already loses
    three digits)."""
    rng = np.random.default_rng(seed)
    A, Bm, b = stable_linear_system(rng, nx, nu)
    th = np.ones(nx) if theta is None else np.asarray(theta, dtype=np.float64)
    ng = nu
    n_dyn = nx * nx + nx * nu + nx
    a = _empty(B, nx, nu, ng, N, n_dyn, 0)
    for i in range(B):
        r = np.random.default_rng([seed, i])
        a["x0"][i] = r.normal(0, 5.0, nx)
        a["Qd"][i] = 2.0 * th
        a["Rd"][i] = 2.0
        a["lo"][i] = -u_max
        a["hi"][i] = u_max
        a["dyn"][i, :nx * nx] = A.ravel()
        a["dyn"][i, nx * nx:nx * nx + nx * nu] = Bm.ravel()
        a["dyn"][i, nx * nx + nx * nu:] = b
    opts = Options(max_sqp=max_sqp, max_admm=max_admm, n_ls=1, early_exit=1, eps_abs=tol, eps_rel=tol, eps_c=tol,
                   rho_max=rho_max)
    pb = ProblemBatch(nx, nu, ng, N, np.full(B, N, np.int32), np.full(B, MODEL_LINEAR, np.int32),
                      opts=opts, name=f"linear_rl_B{B}_N{N}_nx{nx}_nu{nu}_umax{u_max:g}", **a)
    pb.extra = dict(A=A, B=Bm, b=b, theta=th, u_max=u_max)
    return pb


# ----------------------------------------------------------------------------
# humanoid standing balance with single-rigid-body MPC (the SRB model of the
# paper's humanoid imitation-learning appendix)
# ----------------------------------------------------------------------------
SRB_MASS = 33.34                         # kg (paper)
SRB_INERTIA = (1.6, 1.4, 0.35)           # kg m^2, body frame, diagonal (not given in the paper)
SRB_COM_HEIGHT = 0.72                    # m above the feet (not given in the paper)
SRB_FOOT_L = (0.0, 0.1, -SRB_COM_HEIGHT)  # contact points from the CoM (not given in the paper)
SRB_FOOT_R = (0.0, -0.1, -SRB_COM_HEIGHT)
SRB_U_MIN = (-240.0, -240.0, 0.0, -240.0, -240.0, 0.0)      # N (paper: friction cone as a box)
SRB_U_MAX = (240.0, 240.0, 400.0, 240.0, 240.0, 400.0)
SRB_THETA = np.log([50.0, 50.0, 100.0, 30.0, 30.0, 10.0, 5.0, 5.0, 5.0, 1.0, 1.0, 1.0])   # synthetic expert


def humanoid(B=100, N=20, seed=1007, theta=None, max_sqp=5, max_admm=100, dt=0.025) -> ProblemBatch:
    """Standing balance by SRB MPC: state (p, Theta (ZYX roll, pitch, yaw), v,
    omega) in R^12, control the two foot forces (f_L, f_R) in the world frame,
    RK4 at dt = 0.025, horizon N = 20.  Stage cost (x - x_ref)' Q(theta)
    (x - x_ref) + (u - u_ref)' R (u - u_ref) with Q = diag(exp(theta)) and R =
    1e-3 I (written with the 1/2 of the cost convention: Qd = 2 exp(theta), Rd
    = 2e-3); x_ref the standing pose (CoM at SRB_COM_HEIGHT above the origin,
    level, at rest), u_ref = m g / 2 upward on each foot; the friction cone as
    the paper's box on the forces.  x0 = the standing pose perturbed uniformly
    (position 3 cm, angles 0.1 rad, velocity 0.2 m/s, angular rate 0.5 rad/s).
    theta defaults to SRB_THETA (one vector for every instance; a [B, 12] array
    gives one per instance)."""
    nx, nu, ng = 12, 6, 6
    n_dyn = 12
    th = np.broadcast_to(SRB_THETA if theta is None else np.asarray(theta, dtype=np.float64), (B, nx))
    a = _empty(B, nx, nu, ng, N, n_dyn, 0)
    a["z_init"] = np.zeros((B, N + 1, nx + nu))
    xref = np.zeros(nx)
    xref[2] = SRB_COM_HEIGHT
    uref = np.array([0.0, 0.0, 0.5 * SRB_MASS * GRAVITY] * 2)
    for i in range(B):
        r = np.random.default_rng([seed, i])
        a["x0"][i] = xref + r.uniform(-1, 1, nx) * np.repeat([0.03, 0.1, 0.2, 0.5], 3)
        a["Qd"][i, :, :] = 2.0 * np.exp(th[i])
        a["Rd"][i, :, :] = 2e-3
        a["ref"][i, :, :nx] = xref
        a["ref"][i, :, nx:] = uref
        a["lo"][i, :, :] = SRB_U_MIN
        a["hi"][i, :, :] = SRB_U_MAX
        a["dyn"][i] = [dt, SRB_MASS, *SRB_INERTIA, *SRB_FOOT_L, *SRB_FOOT_R, GRAVITY]
        a["z_init"][i, :, :nx] = a["x0"][i]
        a["z_init"][i, :, nx:] = uref
    opts = Options(max_sqp=max_sqp, max_admm=max_admm)
    pb = ProblemBatch(nx, nu, ng, N, np.full(B, N, np.int32), np.full(B, MODEL_SRB, np.int32),
                      opts=opts, name=f"humanoid_B{B}_N{N}", **a)
    pb.extra = dict(theta=np.array(th), xref=xref, uref=uref)
    return pb
