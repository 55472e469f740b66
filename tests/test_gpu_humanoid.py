"""The single-rigid-body humanoid (the SRB model of the paper's humanoid
imitation-learning appendix: nx = 12, nu = 6, RK4 at dt = 0.025, N = 20, box
on the foot forces) on the generic kernel, against the FP64 oracle:

* the RK4 rollout of the initial guess (no SQP step);
* 5 SQP x 100 ADMM at equal counts (sensitivity mode of test_gpu_parity);
* the backward at the oracle's solution, per parameter;
* the gradient of an imitation loss with respect to the log-space cost weights
  theta (Q = diag(exp theta)) through TmpcFunction, against central finite
  differences (h = 1e-3) of the same loss with every solve by the oracle.
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


def test_humanoid_rollout_matches_oracle():
    from paper_2606_24039_gb300 import Solver
    pb = w.humanoid(B=6, max_sqp=0, max_admm=1)
    pb.z_init = None
    s = Solver.from_batch(pb, device="cuda")
    sol = s.tmpc_solve(s.x0)
    torch.cuda.synchronize()
    z = sol["z"].cpu().numpy()
    for i in range(pb.B):
        assert _rel(z[i], osqp.rollout(pb.instance(i))) <= 1e-5, i


def test_humanoid_matches_oracle_at_equal_counts():
    import test_gpu_parity as P
    pb = w.humanoid(B=8)
    s, sol, _ = P._run(pb)
    P._compare(pb, sol, range(pb.B), sensitivity=True)
    assert np.all(np.isin(sol["status"], (0, 1)))


def test_humanoid_backward_on_oracle_point():
    from paper_2606_24039_gb300 import Solver
    import test_gpu_parity as P
    pb = w.humanoid(B=3)
    s = Solver.from_batch(pb, device="cuda")
    refs = [osqp.solve(pb.instance(i), pb.opts) for i in range(pb.B)]
    sol = {}
    for k, kk in (("z", "z"), ("xi", "xi"), ("y_eq", "yf"), ("y_ineq", "yg")):
        sol[k] = torch.tensor(np.stack([r[kk] for r in refs]), dtype=torch.float32, device="cuda")
    sol["status"] = torch.zeros(pb.B, dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(17)
    dLdz = rng.normal(size=(pb.B, pb.N_max + 1, pb.n))
    g = s.tmpc_backward(s.x0, sol, torch.tensor(dLdz, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    keys = ("x0", "Qd", "Rd", "ref", "lin", "lo", "hi")
    for i in range(pb.B):
        inst = {k: (v.astype(np.float32).astype(np.float64) if isinstance(v, np.ndarray) and v.dtype == np.float64
                    else v) for k, v in pb.instance(i).items()}
        point = {k: np.asarray(sol[kk][i].cpu().numpy(), dtype=np.float64) for k, kk in
                 (("z", "z"), ("xi", "xi"), ("yf", "y_eq"), ("yg", "y_ineq"))}
        gr, _ = obwd.backward(inst, point, dLdz[i].astype(np.float64), eps_g=pb.opts.eps_g)
        scale = max(np.linalg.norm(gr[k]) for k in keys)
        for k in keys:
            ga = g[k][i].cpu().numpy().reshape(gr[k].shape)
            assert P._grad_rel(ga.reshape(-1), gr[k].reshape(-1), scale) < P.GRAD_TOL, (i, k)


def _imitation_loss_oracle(pb, theta, u_exp, opts):
    """sum_i 1/N sum_t ||u_t(theta; x0_i) - u_exp_t||^2, every solve by the oracle."""
    L, acts = 0.0, []
    for i in range(pb.B):
        inst = pb.instance(i)
        inst["Qd"] = np.tile(2.0 * np.exp(theta), (pb.N_max + 1, 1))
        o = osqp.solve(inst, opts)
        lw, up, _ = obwd.active_set(inst, o["z"], o["xi"], o["yg"], pb.opts.eps_g)
        acts.append(np.concatenate([lw.reshape(-1), up.reshape(-1)]))
        u = o["z"][:pb.N_max, pb.nx:]
        L += float(np.sum((u - u_exp[i]) ** 2)) / pb.N_max
    return L, acts


def test_imitation_gradient_through_autograd_matches_finite_differences():
    """B = 4 demonstrations by the oracle at the expert weights; a student theta
    off the expert's; the gradient of the imitation loss by autograd through
    TmpcFunction (Qd = 2 exp(theta)) against the oracle's central differences
    along three random directions (skipped where an active set changes within
    +-h)."""
    from paper_2606_24039_gb300 import Solver, solve_ocp
    pb = w.humanoid(B=4, max_sqp=10, max_admm=300)
    tight = dataclasses.replace(pb.opts, eps_abs=1e-10, eps_rel=1e-10, eps_c=1e-10, max_admm=20000, max_sqp=30,
                                early_exit=1)
    u_exp = []
    for i in range(pb.B):
        u_exp.append(osqp.solve(pb.instance(i), tight)["z"][:pb.N_max, pb.nx:])
    rng = np.random.default_rng(21)
    th0 = w.SRB_THETA + rng.uniform(-0.5, 0.5, 12)
    s = Solver.from_batch(pb, device="cuda")
    theta = torch.tensor(th0, dtype=torch.float32, device="cuda", requires_grad=True)
    f = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    Qd = (2.0 * torch.exp(theta))[None, None, :].expand(pb.B, pb.N_max + 1, pb.nx).contiguous()
    z, _, status = solve_ocp(s, f(pb.x0), Qd, f(pb.Rd), f(pb.ref), f(pb.lo), f(pb.hi))
    assert torch.all((status == 0) | (status == 1))
    loss = ((z[:, :pb.N_max, pb.nx:] - f(np.stack(u_exp))) ** 2).sum() / pb.N_max
    loss.backward()
    g = theta.grad.cpu().double().numpy()
    h = 1e-3
    _, base = _imitation_loss_oracle(pb, th0, u_exp, tight)
    checked = 0
    for _ in range(3):
        d = rng.normal(size=12)
        d /= np.linalg.norm(d)
        Lp, ap = _imitation_loss_oracle(pb, th0 + h * d, u_exp, tight)
        Lm, am = _imitation_loss_oracle(pb, th0 - h * d, u_exp, tight)
        if not all(np.array_equal(p, q) and np.array_equal(p, r) for p, q, r in zip(ap, am, base)):
            continue
        fd = (Lp - Lm) / (2 * h)
        assert abs(float(g @ d) - fd) <= 1e-2 * max(abs(fd), 1e-3 * np.linalg.norm(g)), (float(g @ d), fd)
        checked += 1
    assert checked >= 1
