"""GPU parity at the shapes of the paper's workloads that the basic parity
tests do not reach: the implicit-midpoint Newton rollout of the racing model
(Appendix A, Remark A1), the backward pass at the tracking dimensions
(nx = 48, nu = 20, N = 32) on the GPU's own forward output, and the
differentiable layer (torch.autograd.Function) driven by a cost MLP, checked
against the FP64 oracle's gradient chained through the same MLP and against
central finite differences (h = 1e-3) of the oracle.

Tolerances: relative solution error 1e-4 (infinity norm, scale max(1, |z|)),
gradients 1e-3 relative (2-norm, with a floor of 1e-3 of the instance's
gradient scale for gradients that vanish in exact arithmetic).
"""
import dataclasses

import numpy as np
import pytest
import torch

import workloads as w
from oracle import backward as obwd
from oracle import sqp as osqp

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4
GRAD_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_24039_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


def _grad_rel(a, b, scale):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-3 * scale, 1e-12))


# ---------------------------------------------------------------------------
# Newton rollout of the implicit midpoint model (initial guess of Algorithm 1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("solver", [1, 2, 4], ids=["generic", "smem_cr", "warp_ldl"])
def test_newton_rollout_matches_oracle(solver):
    """Instances without an initial guess start from the rollout of the
    reference controls, each x_{t+1} found by 3 Newton steps on the implicit
    midpoint residual from an explicit Euler step.  With no SQP step the
    returned trajectory is that rollout (bicycle at N = 50 on the racing
    tracks, the double integrator and the quadrotor by their explicit maps)."""
    from paper_2606_24039_gb300 import Solver
    pb = w.uneven(B=12, N_lo=10, N_hi=50, seed=91, max_sqp=0, max_admm=1)
    pb.z_init = None
    s = Solver.from_batch(pb, device="cuda", solver=solver)
    sol = s.tmpc_solve(s.x0)
    torch.cuda.synchronize()
    z = sol["z"].cpu().numpy()
    assert np.all(sol["stats"].cpu().numpy()[:, 0] == 0)
    n_bike = 0
    for i in range(pb.B):
        inst = pb.instance(i)
        n = inst["nx"] + inst["nu"]
        ref = osqp.rollout(inst, newton_steps=pb.opts.newton_steps)
        assert _rel(z[i, :inst["N"] + 1, :n], ref) <= REL_TOL, (i, inst["model"])
        n_bike += inst["model"] == w.MODEL_BICYCLE
    assert n_bike >= 3


@pytest.mark.parametrize("solver", [1, 2], ids=["generic", "smem_cr"])
def test_racing_from_the_newton_rollout(solver):
    """Two SQP steps of short racing instances that start from the rollout
    (no centreline guess): the QP built at the rollout and the step taken
    match the oracle at equal iteration counts."""
    from paper_2606_24039_gb300 import Solver
    pb = w.racing(B=6, N=12, max_sqp=1, max_admm=300)
    pb.z_init = None
    s = Solver.from_batch(pb, device="cuda", solver=solver)
    sol = s.tmpc_solve(s.x0)
    torch.cuda.synchronize()
    z = sol["z"].cpu().numpy()
    st = sol["stats"].cpu().numpy()
    for i in range(pb.B):
        o = osqp.solve(pb.instance(i), pb.opts)
        assert st[i, 1] == o["stats"]["admm_iters"]
        assert st[i, 7] == o["history"][0]["alpha"], i
        assert _rel(z[i], o["z"]) <= REL_TOL, (i, _rel(z[i], o["z"]))


# ---------------------------------------------------------------------------
# backward at the tracking dimensions, on the GPU's own forward output
# ---------------------------------------------------------------------------
def _rounded_to_fp32(inst):
    """The instance with every array rounded to FP32, as the GPU receives it (an
    ill-conditioned active-set KKT system amplifies an input difference of one
    FP32 rounding far beyond the gradient bar)."""
    return {k: (v.astype(np.float32).astype(np.float64) if isinstance(v, np.ndarray) and v.dtype == np.float64 else v)
            for k, v in inst.items()}


def _as_oracle_solution(sol, i, inst):
    T, n, nx, ng = inst["N"] + 1, inst["nx"] + inst["nu"], inst["nx"], inst["ng"]
    g = lambda k, m: sol[k][i, :T, :m].cpu().numpy().astype(np.float64)
    return dict(z=g("z", n), xi=g("xi", ng), yf=g("y_eq", nx), yg=g("y_ineq", ng))


def test_backward_tracking_dims_on_gpu_forward():
    """nx = 48, nu = 20, N = 32 (the tracking workload's dims, n = 68): the GPU
    forward solution (400 ADMM iterations) is the point; the GPU backward
    and the oracle's active-set KKT solve at that same point agree per
    parameter, and the active sets agree."""
    from paper_2606_24039_gb300 import Solver
    pb = w.tracking(B=4, max_admm=400)
    s = Solver.from_batch(pb, device="cuda")
    sol = s.tmpc_solve(s.x0)
    rng = np.random.default_rng(17)
    dLdz = rng.normal(size=(pb.B, pb.N_max + 1, pb.n))
    g = s.tmpc_backward(s.x0, sol, torch.tensor(dLdz, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    keys = ("x0", "Qd", "Rd", "ref", "lin", "lo", "hi")
    nact = 0
    for i in range(pb.B):
        inst = pb.instance(i)
        point = _as_oracle_solution(sol, i, inst)
        gr, info = obwd.backward(inst, point, dLdz[i], eps_g=pb.opts.eps_g)
        assert not info["singular"]
        nact += int(info["lower"].sum() + info["upper"].sum())
        scale = max(np.linalg.norm(gr[k]) for k in keys)
        for k in keys:   # every instance spans the whole layout (N = N_max, model dims = layout dims)
            rel = _grad_rel(g[k][i].cpu().numpy().reshape(-1), gr[k].reshape(-1), scale)
            assert rel < GRAD_TOL, (i, k, rel)
    assert nact > 0


# ---------------------------------------------------------------------------
# the differentiable layer driven by a cost MLP (tracking workload)
# ---------------------------------------------------------------------------
def _mlp_torch(params, ctx):
    h = ctx
    L = len(params) // 2
    for k in range(L):
        h = h @ params[2 * k].T + params[2 * k + 1]
        if k < L - 1:
            h = torch.tanh(h)
    return h


def _tracking_loss_np(z, ref, nx, N):
    """L = 1/(N+1) sum_t ||x_t - r_t||^2 + 1e-3 ||u_t||^2 and dL/dz."""
    dx = z[:, :nx] - ref[:, :nx]
    u = z[:, nx:]
    L = float(np.sum(dx * dx) / (N + 1) + 1e-3 * np.sum(u * u))
    g = np.concatenate([2.0 * dx / (N + 1), 2e-3 * u], axis=1)
    return L, g


def _oracle_point(pb, i, out64, x0, lo, hi, opts):
    inst = pb.instance(i)
    nx, T = pb.nx, pb.N_max + 1
    inst["Qd"] = np.tile(np.exp(out64[i, :nx]), (T, 1))
    inst["Rd"] = np.tile(w.R_SCALE_TRACKING * np.exp(out64[i, nx:]), (T, 1))
    inst["x0"] = x0[i].copy()
    inst["lo"] = lo[i].copy()
    inst["hi"] = hi[i].copy()
    return inst, osqp.solve(inst, opts)


def _oracle_loss(pb, params64, ctx, x0, lo, hi, opts):
    out64 = w.mlp_forward_np(params64, ctx)
    tot = 0.0
    acts = []
    for i in range(pb.B):
        inst, o = _oracle_point(pb, i, out64, x0, lo, hi, opts)
        L, _ = _tracking_loss_np(o["z"], inst["ref"], pb.nx, inst["N"])
        tot += L
        lw, up, _ = obwd.active_set(inst, o["z"], o["xi"], o["yg"], opts.eps_g)
        acts.append(np.concatenate([lw.reshape(-1), up.reshape(-1)]))
    return tot, acts


def test_autograd_function_through_cost_mlp():
    """Tracking dims (nx = 48, nu = 20, N = 32), cost weights Q = exp(o_x),
    R = 0.1 exp(o_u) with o = MLP(context), loss 1/(N+1) sum ||x - r||^2 +
    1e-3 ||u||^2.  The gradients of torch autograd through TmpcFunction
    (GPU forward and backward) with respect to the MLP parameters, x0 and the
    bounds equal the FP64 oracle's active-set gradient chained through the
    same MLP, and the oracle's gradient equals its own central finite
    differences (h = 1e-3) along random directions of the MLP parameters,
    of x0 and of the control bound u_max (instances whose active set
    changes at +-h are excluded from the difference quotient)."""
    from paper_2606_24039_gb300 import Solver, solve_ocp
    pb = w.tracking(B=4, max_admm=400)
    nx, nu, T, N = pb.nx, pb.nu, pb.N_max + 1, pb.N_max
    mlp, ctx = pb.extra["mlp"], pb.extra["ctx"][:pb.B]
    s = Solver.from_batch(pb, device="cuda")
    params = [torch.tensor(a, dtype=torch.float32, device="cuda", requires_grad=True) for a in mlp]
    ctx_t = torch.tensor(ctx, dtype=torch.float32, device="cuda")
    x0 = s.x0.clone().requires_grad_(True)
    lo = torch.tensor(pb.lo, dtype=torch.float32, device="cuda", requires_grad=True)
    hi = torch.tensor(pb.hi, dtype=torch.float32, device="cuda", requires_grad=True)
    ref = torch.tensor(pb.ref, dtype=torch.float32, device="cuda")
    out = _mlp_torch(params, ctx_t)
    Qd = torch.exp(out[:, :nx])[:, None, :].expand(pb.B, T, nx).contiguous()
    Rd = (w.R_SCALE_TRACKING * torch.exp(out[:, nx:]))[:, None, :].expand(pb.B, T, nu).contiguous()
    z, xi, status = solve_ocp(s, x0, Qd, Rd, ref, lo, hi)
    dx = z[:, :, :nx] - ref[:, :, :nx]
    loss = (dx * dx).sum() / (N + 1) + 1e-3 * (z[:, :, nx:] ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    assert torch.all(status != 3)

    # oracle: the same float32 parameters in FP64, converged solves, active-set backward
    opts = dataclasses.replace(pb.opts, max_admm=20000, early_exit=1, eps_abs=1e-11, eps_rel=1e-11)
    p64 = [p.detach().cpu().double().numpy() for p in params]
    x064 = x0.detach().cpu().double().numpy()
    lo64 = lo.detach().cpu().double().numpy()
    hi64 = hi.detach().cpu().double().numpy()
    out64 = w.mlp_forward_np(p64, ctx)
    dL_do = np.zeros((pb.B, nx + nu))
    g_x0 = np.zeros((pb.B, nx))
    g_lo = np.zeros_like(lo64)
    g_hi = np.zeros_like(hi64)
    for i in range(pb.B):
        inst, o = _oracle_point(pb, i, out64, x064, lo64, hi64, opts)
        _, dLdz = _tracking_loss_np(o["z"], inst["ref"], nx, N)
        gr, info = obwd.backward(inst, o, dLdz, eps_g=pb.opts.eps_g)
        assert not info["singular"]
        dL_do[i, :nx] = np.sum(gr["Qd"] * inst["Qd"], axis=0)       # dQ/do = Q
        dL_do[i, nx:] = np.sum(gr["Rd"] * inst["Rd"], axis=0)       # dR/do = R
        g_x0[i], g_lo[i], g_hi[i] = gr["x0"], gr["lo"], gr["hi"]
    pt = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in p64]
    (_mlp_torch(pt, torch.tensor(ctx, dtype=torch.float64)) * torch.tensor(dL_do)).sum().backward()
    g_par = [p.grad.numpy() for p in pt]

    scale = max(np.linalg.norm(g) for g in g_par)
    for k, (pg, og) in enumerate(zip(params, g_par)):
        rel = _grad_rel(pg.grad.cpu().numpy().reshape(-1), og.reshape(-1), scale)
        assert rel < GRAD_TOL, ("mlp parameter", k, rel)
    for name, gpu, ora in (("x0", x0.grad, g_x0), ("lo", lo.grad, g_lo), ("hi", hi.grad, g_hi)):
        for i in range(pb.B):
            sc = max(np.linalg.norm(g_x0[i]), np.linalg.norm(g_lo[i]), np.linalg.norm(g_hi[i]))
            rel = _grad_rel(gpu[i].cpu().numpy().reshape(-1), ora[i].reshape(-1), sc)
            assert rel < GRAD_TOL, (name, i, rel)

    # central finite differences of the oracle (h = 1e-3) along random directions
    h = 1e-3
    rng = np.random.default_rng(23)
    base_acts = _oracle_loss(pb, p64, ctx, x064, lo64, hi64, opts)[1]

    def fd(pp, xp, lp, hp, pm, xm, lm, hm):
        Lp, ap = _oracle_loss(pb, pp, ctx, xp, lp, hp, opts)
        Lm, am = _oracle_loss(pb, pm, ctx, xm, lm, hm, opts)
        same = all(np.array_equal(a, b) and np.array_equal(a, c) for a, b, c in zip(ap, am, base_acts))
        return (Lp - Lm) / (2 * h), same

    d = [rng.normal(size=a.shape) for a in p64]
    nrm = np.sqrt(sum(np.sum(v * v) for v in d))
    d = [v / nrm for v in d]
    q, same = fd([a + h * v for a, v in zip(p64, d)], x064, lo64, hi64,
                 [a - h * v for a, v in zip(p64, d)], x064, lo64, hi64)
    ana = sum(float(np.sum(g * v)) for g, v in zip(g_par, d))
    gpu = sum(float(np.sum(p.grad.cpu().double().numpy() * v)) for p, v in zip(params, d))
    if same:
        assert abs(ana - q) <= 1e-3 * max(abs(q), 1e-3 * scale), (ana, q)
        assert abs(gpu - q) <= 2e-3 * max(abs(q), 1e-3 * scale), (gpu, q)
    dx0 = rng.normal(size=x064.shape)
    dx0 /= np.linalg.norm(dx0)
    q, same_x = fd(p64, x064 + h * dx0, lo64, hi64, p64, x064 - h * dx0, lo64, hi64)
    if same_x:
        assert abs(float(np.sum(g_x0 * dx0)) - q) <= 1e-3 * max(abs(q), 1e-6), (np.sum(g_x0 * dx0), q)
        assert abs(float(np.sum(x0.grad.cpu().double().numpy() * dx0)) - q) <= 2e-3 * max(abs(q), 1e-6)
    # u_max: hi = +u_max, lo = -u_max on every control row
    q, same_u = fd(p64, x064, lo64 - h, hi64 + h, p64, x064, lo64 + h, hi64 - h)
    du_ora = float(np.sum(g_hi) - np.sum(g_lo))
    du_gpu = float(hi.grad.sum().item() - lo.grad.sum().item())
    if same_u:
        assert abs(du_ora - q) <= 1e-3 * max(abs(q), 1e-6), (du_ora, q)
        assert abs(du_gpu - q) <= 2e-3 * max(abs(q), 1e-6), (du_gpu, q)
    assert same or same_x or same_u   # at least one difference quotient was taken


# ---------------------------------------------------------------------------
# backward of the uneven batch at full size, on the GPU's own forward output
# ---------------------------------------------------------------------------
def test_backward_uneven_full_batch_on_gpu_forward():
    """The uneven batch (4096 instances, N in 10..200, three models, 10 SQP x 50
    ADMM) forward and backward in the launch configuration the benchmark times;
    16 sampled instances: the direct FP64 adjoint solve of the small models and
    the oracle's sparse LU of the same active-set KKT system, built from the
    same (FP32) parameters at the GPU's forward point, agree per parameter
    (instances whose KKT matrix the oracle finds singular are compared after
    the same -1e-10 regularisation)."""
    from paper_2606_24039_gb300 import Solver
    pb = w.uneven(B=4096)
    s = Solver.from_batch(pb, device="cuda")
    sol = s.tmpc_solve(s.x0, z_init=s.z_init)
    rng = np.random.default_rng(3)
    dLdz = rng.normal(size=(pb.B, pb.N_max + 1, pb.n)).astype(np.float32)
    g = s.tmpc_backward(s.x0, sol, torch.tensor(dLdz, device="cuda"))
    torch.cuda.synchronize()
    keys = ("x0", "Qd", "Rd", "Wd", "ref", "lin", "lo", "hi", "gamma2", "gamma1")
    idx = np.random.default_rng(8).choice(pb.B, 16, replace=False)
    worst = []
    for i in idx:
        inst = _rounded_to_fp32(pb.instance(i))   # the parameters the GPU solved with
        T, n, nx, nu, ng = inst["N"] + 1, inst["nx"] + inst["nu"], inst["nx"], inst["nu"], inst["ng"]
        p = _as_oracle_solution(sol, i, inst)
        gr, info = obwd.backward(inst, p, dLdz[i, :T, :n].astype(np.float64), eps_g=pb.opts.eps_g)
        cut = {"x0": (nx,), "Qd": (T, nx), "Rd": (T, nu), "Wd": (nu,), "ref": (T, n), "lin": (T, n),
               "lo": (T, ng), "hi": (T, ng), "gamma2": (ng,), "gamma1": (ng,)}
        scale = max(np.linalg.norm(gr[k]) for k in keys)
        for k in keys:
            ga = g[k][i].cpu().numpy()[tuple(slice(0, m) for m in cut[k])]
            rel = _grad_rel(ga.reshape(-1), gr[k].reshape(-1), scale)
            worst.append((rel, int(i), k, bool(info["singular"])))
            assert rel < GRAD_TOL, (int(i), inst["model"], k, rel, info["singular"])


# ---------------------------------------------------------------------------
# the long-horizon workload itself: 8 racing instances of N = 8192 (dt = 0.01)
# ---------------------------------------------------------------------------
def test_long_horizon_at_full_size():
    """N = 8192 in the launch configuration the benchmark times (one 16-CTA
    cluster per instance).  (a) 5 SQP x 100 ADMM: every instance ends finite,
    OK or at the iteration caps, with its primal residual below the oracle's
    starting level (an FP32 solve that no longer tracks S would diverge here).
    (b) The fixed-count comparison is inconclusive at this size: the QP is far
    from converged after 100 iterations and 1e-7 input perturbations move the
    FP64 result by ~5e-2, so the forward is compared under a converged QP: one
    SQP step with 3000 ADMM iterations, the same line-search step as the oracle
    and the solution within 1e-4, on two instances.  (c) The backward with
    respect to every parameter (the cost weights included) at the oracle's
    point of instance 1, per parameter, within 1e-3."""
    from paper_2606_24039_gb300 import Solver
    from paper_2606_24039_gb300._abi import ls_history
    pb = w.long_horizon()
    s = Solver.from_batch(pb, device="cuda")
    sol = s.tmpc_solve(s.x0, z_init=s.z_init)
    torch.cuda.synchronize()
    st = sol["stats"].cpu().numpy()
    assert np.all(np.isin(sol["status"].cpu().numpy(), (0, 1)))
    assert np.all(np.isfinite(sol["z"].cpu().numpy()))
    assert np.all(st[:, 2] < 10.0), st[:, 2]
    pc = w.long_horizon(max_sqp=1, max_admm=3000)
    sc = Solver.from_batch(pc, device="cuda")
    solc = sc.tmpc_solve(sc.x0, z_init=sc.z_init)
    torch.cuda.synchronize()
    zc, stc = solc["z"].cpu().numpy(), solc["stats"].cpu().numpy()
    for i in (0, 1):
        o = osqp.solve(pc.instance(i), pc.opts, record=True)
        assert ls_history(stc[i], stc[i][0]) == [h.get("alpha") for h in o["history"]], i
        assert _rel(zc[i], o["z"]) <= REL_TOL, (i, _rel(zc[i], o["z"]))
    i = 1
    own = osqp.solve(pb.instance(i), pb.opts)
    sol2 = {}
    for k, kk in (("z", "z"), ("xi", "xi"), ("y_eq", "yf"), ("y_ineq", "yg")):
        arr = np.zeros((pb.B,) + own[kk].shape, np.float32)
        arr[i] = own[kk]
        sol2[k] = torch.tensor(arr, device="cuda")
    sol2["status"] = torch.zeros(pb.B, dtype=torch.int32, device="cuda")
    dLdz = np.random.default_rng(13).normal(size=(pb.B, pb.N_max + 1, pb.n))
    g = s.tmpc_backward(s.x0, sol2, torch.tensor(dLdz, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    inst = _rounded_to_fp32(pb.instance(i))
    point = {k: np.asarray(sol2[kk][i].cpu().numpy(), dtype=np.float64) for k, kk in
             (("z", "z"), ("xi", "xi"), ("yf", "y_eq"), ("yg", "y_ineq"))}
    gr, _ = obwd.backward(inst, point, dLdz[i].astype(np.float64), eps_g=pb.opts.eps_g)
    T = pb.N_max + 1
    keys = {"x0": (6,), "Qd": (T, 6), "Rd": (T, 2), "Wd": (2,), "ref": (T, 8), "lin": (T, 8), "lo": (T, 5),
            "hi": (T, 5)}
    scale = max(np.linalg.norm(gr[k]) for k in keys)
    for k, cut in keys.items():
        ga = g[k][i].cpu().numpy()[tuple(slice(0, m) for m in cut)]
        assert _grad_rel(ga.reshape(-1), gr[k].reshape(-1), scale) < GRAD_TOL, k
