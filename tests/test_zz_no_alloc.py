"""The no-allocation entry point tmpc_solve_static (collected last on purpose:
it must pass alone and after every other test in the same process)."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as w

pytestmark = pytest.mark.gpu


def _inputs(pb):
    from paper_2606_24039_gb300 import tensors_from_batch
    t = tensors_from_batch(pb, "cuda")
    dims = dict(batch=pb.B, N_max=pb.N_max, nx=pb.nx, nu=pb.nu, ng=pb.ng, n_dyn=pb.n_dyn, n_track=pb.n_track)
    return t, dims


def _zeroed_like(sol):
    return {k: torch.zeros_like(v) for k, v in sol.items()}


@pytest.mark.parametrize("make", [
    lambda: w.double_integrator(B=6, N=20, max_admm=200),
    lambda: w.racing(B=8, N=30, max_sqp=3, max_admm=40),
], ids=["double_integrator", "racing"])
def test_static_entry_matches_handle_entry_twice(make):
    from paper_2606_24039_gb300 import Solver, options_from, tmpc_solve_static
    pb = make()
    if pb.model[0] == w.MODEL_DI:
        pb.N[:] = [20, 1, 2, 7, 13, 19]
    t, dims = _inputs(pb)
    s = Solver.from_batch(pb, device="cuda", solver=1)       # existing entry, same kernel
    ref = s.tmpc_solve(s.x0, z_init=s.z_init)
    opts = options_from(pb.opts, solver=1)
    for _ in range(2):                                       # two calls in a row
        out = _zeroed_like(ref)
        if t["z_init"] is not None:
            out["z"].copy_(t["z_init"])
        tmpc_solve_static(dims, t, t["x0"], out, opts, warm_start=t["z_init"] is not None)
        torch.cuda.synchronize()
        # same kernel and arithmetic per instance, whatever order the queue hands them out in
        for k in ("z", "xi", "y_eq", "y_ineq", "stats", "status"):
            assert torch.equal(out[k], ref[k]), k


def test_static_entry_allocates_no_device_memory():
    """The defining property: after a first call (which looks up the scratch
    address once), further calls change neither the device's free memory nor
    torch's allocator."""
    from paper_2606_24039_gb300 import options_from, tmpc_solve_static
    pb = w.racing(B=8, N=30, max_sqp=2, max_admm=30)
    t, dims = _inputs(pb)
    opts = options_from(pb.opts, solver=1)
    out = {k: torch.zeros((pb.B,) + tuple(v.shape[1:]), device="cuda") for k, v in
           (("z", t["z_init"]), ("xi", t["lo"]), ("y_eq", t["Qd"]), ("y_ineq", t["lo"]))}
    out["status"] = torch.zeros(pb.B, dtype=torch.int32, device="cuda")
    out["stats"] = torch.zeros((pb.B, 10), device="cuda")
    tmpc_solve_static(dims, t, t["x0"], out, opts)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        tmpc_solve_static(dims, t, t["x0"], out, opts)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0
    assert np.all(np.isin(out["status"].cpu().numpy(), (0, 1)))


def test_handle_still_launches_after_a_smaller_static_call():
    """A static call with a smaller shared-memory need must not lower the launch
    limit a handle set up for a larger one relies on (generic kernel, ADMM
    vectors in shared memory above 48 KB in both calls)."""
    from paper_2606_24039_gb300 import Solver, options_from, tmpc_solve_static
    big = w.racing(B=4, N=200, max_sqp=2, max_admm=20)
    s = Solver.from_batch(big, device="cuda", solver=1)
    first = {k: v.clone() for k, v in s.tmpc_solve(s.x0, z_init=s.z_init).items()}
    torch.cuda.synchronize()
    small = w.racing(B=4, N=170, max_sqp=2, max_admm=20)
    t, dims = _inputs(small)
    out = {k: torch.zeros((small.B,) + tuple(v.shape[1:]), device="cuda") for k, v in
           (("z", t["z_init"]), ("xi", t["lo"]), ("y_eq", t["Qd"]), ("y_ineq", t["lo"]))}
    out["z"].copy_(t["z_init"])
    out["status"] = torch.zeros(small.B, dtype=torch.int32, device="cuda")
    out["stats"] = None
    tmpc_solve_static(dims, t, t["x0"], out, options_from(small.opts, solver=1), warm_start=True)
    torch.cuda.synchronize()
    again = s.tmpc_solve(s.x0, z_init=s.z_init)
    torch.cuda.synchronize()
    for k in ("z", "xi", "y_eq", "y_ineq", "status", "stats"):
        assert torch.equal(again[k], first[k]), k
    s.close()


def test_static_entry_rejects_a_batch_beyond_the_scratch():
    from paper_2606_24039_gb300 import TmpcError, tmpc_solve_static
    from paper_2606_24039_gb300._abi import STATIC_SCRATCH_BYTES
    pb = w.racing(B=2, N=30, max_sqp=1, max_admm=5)
    t, dims = _inputs(pb)
    dims = dict(dims, batch=4096, N_max=30)    # 4096 x ~50 KB > 64 MiB; nothing is enqueued
    out = {k: torch.zeros(1, device="cuda") for k in ("z", "xi", "y_eq", "y_ineq", "stats")}
    out["status"] = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(TmpcError, match="static scratch holds %d bytes" % STATIC_SCRATCH_BYTES):
        tmpc_solve_static(dims, t, t["x0"], out)


def test_static_entry_marks_out_of_range_instances():
    from paper_2606_24039_gb300 import Solver, options_from, tmpc_solve_static
    pb = w.double_integrator(B=4, N=12, max_admm=50)
    t, dims = _inputs(pb)
    s = Solver.from_batch(pb, device="cuda", solver=1)
    ref = s.tmpc_solve(s.x0)
    t["N"] = torch.tensor([12, 13, 12, 0], dtype=torch.int32, device="cuda")   # 13 > N_max, 0 < 1
    out = {k: torch.full_like(v, 7) for k, v in ref.items()}
    tmpc_solve_static(dims, t, t["x0"], out, options_from(pb.opts, solver=1))
    torch.cuda.synchronize()
    st = out["status"].cpu().numpy()
    assert st[1] == 4 and st[3] == 4
    for i in (1, 3):
        assert torch.count_nonzero(out["z"][i]) == 0 and torch.count_nonzero(out["stats"][i]) == 0
    for i in (0, 2):
        assert st[i] == ref["status"][i].item()
        assert torch.equal(out["z"][i], ref["z"][i])
