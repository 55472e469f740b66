"""Per-instance failure statuses, injected from the host (nothing here can
fault, trap or hang the GPU): a NaN initial state, an indefinite cost that
makes S lose positive definiteness, contradictory bounds, the caller-forced
pivot failure of the options, and bounded waits on the generic kernel's
asynchronous copies cut to one poll.  In every case the other instances of
the batch are unaffected (bit for bit) and the call itself succeeds."""
import numpy as np
import pytest
import torch

import workloads as w

pytestmark = pytest.mark.gpu

OK, MAX_ITER, NOT_PD, NAN, INVALID, TIMEOUT = 0, 1, 2, 3, 4, 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_24039_gb300 import build
    build.build()


def _solve(pb, **over):
    from paper_2606_24039_gb300 import Solver
    s = Solver.from_batch(pb, device="cuda", **over)
    sol = s.tmpc_solve(s.x0, z_init=s.z_init)
    torch.cuda.synchronize()
    return s, {k: v.cpu().numpy() for k, v in sol.items()}, sol


def _others_unchanged(a, b, skip):
    for i in range(len(a["status"])):
        if i in skip:
            continue
        for k in ("z", "xi", "y_eq", "y_ineq", "status", "stats"):
            assert np.array_equal(a[k][i], b[k][i]), (i, k)


SOLVERS = [pytest.param(1, id="generic"), pytest.param(2, id="smem_cr")]


@pytest.mark.parametrize("solver", SOLVERS)
def test_nan_initial_state_is_reported(solver):
    pb = w.uneven(B=8, N_lo=10, N_hi=30, seed=5, max_sqp=2, max_admm=30)
    keep = [i for i in range(pb.B) if pb.model[i] != w.MODEL_BICYCLE]
    _, clean, _ = _solve(pb, solver=solver)
    pb.x0[keep[0], 1] = np.nan
    _, bad, _ = _solve(pb, solver=solver)
    assert bad["status"][keep[0]] == NAN
    _others_unchanged(bad, clean, {keep[0]})


@pytest.mark.parametrize("solver", SOLVERS)
def test_indefinite_cost_is_reported_not_pd(solver):
    """Q = -1e4 on one stage of one instance: a diagonal block of S is not
    positive definite and the block factorisation reports it."""
    pb = w.double_integrator(B=4, N=20, max_admm=60)
    _, clean, _ = _solve(pb, solver=solver)
    pb.Qd[1, 7, :] = -1e4
    _, bad, _ = _solve(pb, solver=solver)
    assert bad["status"][1] == NOT_PD
    _others_unchanged(bad, clean, {1})


@pytest.mark.parametrize("solver", SOLVERS)
def test_contradictory_bounds_end_unconverged_and_finite(solver):
    """lo > hi on the control rows of one instance: the QP is infeasible, the
    projection keeps z_g at the upper bound and ADMM cannot converge."""
    pb = w.double_integrator(B=4, N=20, max_admm=100)
    _, clean, _ = _solve(pb, solver=solver)
    pb.lo[2, :, 0:2] = 2.0
    pb.hi[2, :, 0:2] = 1.0
    _, bad, _ = _solve(pb, solver=solver)
    assert bad["status"][2] == MAX_ITER
    assert np.all(np.isfinite(bad["z"][2]))
    _others_unchanged(bad, clean, {2})


@pytest.mark.parametrize("solver", SOLVERS + [pytest.param(7, id="plain")])
def test_forced_pivot_failure_is_honoured(solver):
    """force_pivot_failure = i + 1: instance i is reported NOT_PD by the forward
    and the backward pass; its arithmetic and every other instance are unchanged."""
    pb = w.racing(B=5, N=20, max_sqp=2, max_admm=30)
    s0, clean, _ = _solve(pb, solver=solver)
    s1, bad, sol_d = _solve(pb, solver=solver, force_pivot_failure=4)
    assert bad["status"][3] == NOT_PD
    for k in ("z", "xi", "y_eq", "y_ineq", "stats"):
        assert np.array_equal(bad[k][3], clean[k][3]), k
    _others_unchanged(bad, clean, {3})
    if solver != 7:
        sol_d["status"].zero_()
        dz = torch.ones_like(sol_d["z"])
        s1.tmpc_backward(s1.x0, sol_d, dz)
        torch.cuda.synchronize()
        st = sol_d["status"].cpu().numpy()
        assert st[3] == NOT_PD and np.all(np.delete(st, 3) != NOT_PD)


def test_bounded_wait_gives_up_and_the_handle_recovers():
    """Generic kernel on the tracking dims (its factor blocks stream through
    shared memory by asynchronous bulk copies): when every wait gives up (the
    caller-forced timeout), the instances finish on global-memory reads of the
    same blocks (bit-identical results) and report TIMEOUT; the copies still in
    flight are waited for before the buffers are reused, so the next solve on
    the same handle with the default waits is clean again.  One poll per wait
    (wait_polls = 1) gives the same results whichever way each wait ends."""
    from paper_2606_24039_gb300 import options_from
    pb = w.tracking(B=6, max_admm=60)
    s, clean, _ = _solve(pb)
    s2, cut, _ = _solve(pb, force_wait_timeout=1)
    assert np.all(cut["status"] == TIMEOUT)
    for k in ("z", "xi", "y_eq", "y_ineq"):
        assert np.array_equal(cut[k], clean[k]), k
    s2.tmpc_set_options(options_from(pb.opts))
    again = s2.tmpc_solve(s2.x0)
    torch.cuda.synchronize()
    for k in ("z", "xi", "y_eq", "y_ineq", "status", "stats"):
        assert np.array_equal(again[k].cpu().numpy(), clean[k]), k
    s3, one, _ = _solve(pb, wait_polls=1)
    assert np.all(np.isin(one["status"], (TIMEOUT, clean["status"][0])))
    for k in ("z", "xi", "y_eq", "y_ineq"):
        assert np.array_equal(one[k], clean[k]), k
