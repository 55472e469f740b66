"""The linear-system RL problem family (Section IV, linear-system RL scaling):
x+ = A x + B u + b with a control box, stage cost x'Qx + ||u||^2, Q = diag(theta).

* parity of the CUDA path with the FP64 oracle at equal iteration counts
  (affine dynamics, the nominal dims nx = 8, nu = 4, N = 40, and n = 24);
* at the paper's tolerance (early exit at 1e-5, at most 1e3 ADMM iterations)
  every instance ends finite and within 1e-4 of the converged FP64 solution;
* the reward gradient through closed-loop MPC rollouts (torch autograd over
  TmpcFunction) matches central finite differences (h = 1e-3) of the same
  closed loop run with the FP64 oracle.
"""
import dataclasses

import numpy as np
import pytest
import torch

import workloads as w
from oracle import backward as obwd
from oracle import sqp as osqp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_24039_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


@pytest.mark.parametrize("nx,nu,u_max", [(8, 4, 1.0), (16, 8, 10.0)], ids=["n12_umax1", "n24_umax10"])
def test_linear_rl_matches_oracle_at_equal_counts(nx, nu, u_max):
    from paper_2606_24039_gb300 import Solver
    pb = w.linear_rl(B=4, nx=nx, nu=nu, u_max=u_max, max_sqp=2, max_admm=150)
    pb.opts = dataclasses.replace(pb.opts, early_exit=0)
    s = Solver.from_batch(pb, device="cuda")
    sol = s.tmpc_solve(s.x0)
    torch.cuda.synchronize()
    z = sol["z"].cpu().numpy()
    st = sol["stats"].cpu().numpy()
    for i in range(pb.B):
        o = osqp.solve(pb.instance(i), pb.opts)
        assert st[i, 0] == o["stats"]["sqp_iters"] and st[i, 1] == o["stats"]["admm_iters"]
        assert _rel(z[i], o["z"]) <= 1e-4, (i, _rel(z[i], o["z"]))


def test_linear_rl_at_the_tolerance_matches_the_converged_oracle():
    """Nominal configuration (B = 64, N = 40, nx = 8, nu = 4, u_max = 1) at
    tol = 1e-5: every instance ends finite (OK or at the iteration caps), and its
    solution is within 1e-4 of the oracle's solution converged to 1e-10."""
    from paper_2606_24039_gb300 import Solver
    pb = w.linear_rl(B=64)
    s = Solver.from_batch(pb, device="cuda")
    sol = s.tmpc_solve(s.x0)
    torch.cuda.synchronize()
    status = sol["status"].cpu().numpy()
    assert np.all(np.isin(status, (0, 1))), np.unique(status, return_counts=True)
    z = sol["z"].cpu().numpy()
    tight = dataclasses.replace(pb.opts, eps_abs=1e-10, eps_rel=1e-10, eps_c=1e-10, max_admm=20000, max_sqp=20)
    for i in range(0, pb.B, 16):
        o = osqp.solve(pb.instance(i), tight)
        assert _rel(z[i], o["z"]) <= 1e-4, (i, _rel(z[i], o["z"]))


def _closed_loop_oracle(pb, theta, H):
    """Reward -(sum_k ||x_k||^2 + ||u_k||^2) of H closed-loop steps, every MPC
    solve by the FP64 oracle to 1e-10; also the active sets met on the way."""
    A, Bm, b = pb.extra["A"], pb.extra["B"], pb.extra["b"]
    opts = dataclasses.replace(pb.opts, eps_abs=1e-10, eps_rel=1e-10, eps_c=1e-10, max_admm=20000, max_sqp=20)
    R, acts = 0.0, []
    for i in range(pb.B):
        x = pb.x0[i].copy()
        for _ in range(H):
            inst = pb.instance(i)
            inst["x0"] = x
            inst["Qd"] = np.tile(2.0 * theta, (pb.N_max + 1, 1))
            o = osqp.solve(inst, opts)
            lw, up, _ = obwd.active_set(inst, o["z"], o["xi"], o["yg"], pb.opts.eps_g)
            acts.append(np.concatenate([lw.reshape(-1), up.reshape(-1)]))
            u = o["z"][0, pb.nx:]
            R -= float(x @ x + u @ u)
            x = A @ x + Bm @ u + b
    return R, acts


def test_closed_loop_reward_gradient_matches_finite_differences():
    """H = 5 closed-loop steps of B = 2 episodes (N = 10): the gradient of the
    episode reward with respect to theta = diag(Q), by autograd through the
    GPU solves (the state fed back is differentiable, so the x0 gradient of
    each solve chains the steps), equals the oracle's central differences."""
    from paper_2606_24039_gb300 import Solver, solve_ocp
    H = 5
    pb = w.linear_rl(B=2, N=10)
    nx = pb.nx
    s = Solver.from_batch(pb, device="cuda")
    A = torch.tensor(pb.extra["A"], dtype=torch.float32, device="cuda")
    Bm = torch.tensor(pb.extra["B"], dtype=torch.float32, device="cuda")
    b = torch.tensor(pb.extra["b"], dtype=torch.float32, device="cuda")
    theta = torch.tensor(pb.extra["theta"], dtype=torch.float32, device="cuda", requires_grad=True)
    Rd = torch.tensor(pb.Rd, dtype=torch.float32, device="cuda")
    ref = torch.zeros((pb.B, pb.N_max + 1, pb.n), device="cuda")
    lo = torch.tensor(pb.lo, dtype=torch.float32, device="cuda")
    hi = torch.tensor(pb.hi, dtype=torch.float32, device="cuda")
    x = torch.tensor(pb.x0, dtype=torch.float32, device="cuda")
    reward = torch.zeros((), device="cuda")
    for _ in range(H):
        Qd = (2.0 * theta)[None, None, :].expand(pb.B, pb.N_max + 1, nx).contiguous()
        z, _, status = solve_ocp(s, x, Qd, Rd, ref, lo, hi)
        assert torch.all((status == 0) | (status == 1))
        u = z[:, 0, nx:]
        reward = reward - (x * x).sum() - (u * u).sum()
        x = x @ A.T + u @ Bm.T + b
    reward.backward()
    g = theta.grad.cpu().double().numpy()

    h = 1e-3
    th0 = pb.extra["theta"]
    _, base = _closed_loop_oracle(pb, th0, H)
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(3):
        d = rng.normal(size=nx)
        d /= np.linalg.norm(d)
        Rp, ap = _closed_loop_oracle(pb, th0 + h * d, H)
        Rm, am = _closed_loop_oracle(pb, th0 - h * d, H)
        if not all(np.array_equal(p, q) and np.array_equal(p, r) for p, q, r in zip(ap, am, base)):
            continue    # an active set changes inside +-h: the difference quotient is not a derivative
        fd = (Rp - Rm) / (2 * h)
        assert abs(float(g @ d) - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.linalg.norm(g)), (float(g @ d), fd)
        checked += 1
    assert checked >= 1
