"""The rescaled ADMM (normalised states and controls, Remark 4) on the GPU,
through the C ABI, against the FP64 oracle's rescaled ADMM (oracle.admm
.admm_rescaled, pinned on the CPU by tests/test_oracle_rescale.py):

* ragged double-integrator batches with per-instance, per-component scales
  (shared-memory cyclic reduction, warp LDL', global arenas) and racing with
  the magnitude scales of the workload, at equal iteration counts, residuals
  compared in the scaled units both sides report.  Both are held to the
  sensitivity-mode bar of the parity harness: on these rescaled problems the
  rho rule takes large steps (rho_bar up to 10 on the double integrator) and
  the fixed-count solution of the FP64 oracle itself moves by up to 2.4e-3
  (double integrator, 200 ADMM iterations) and 3e-4 (racing, 1 x 100) under
  FP32 rounding of its inputs and factorisations, so a strict 1e-4 bar would
  test rounding, not the method;
* the launch forms agree bit for bit with scales (shared vs global arenas,
  persistent vs plain per-phase), unit scales change nothing, the cluster team
  matches the single CTA, and the host-memory entry point equals the device one;
* a scale on an instance the generic kernel would run is refused before any
  work is enqueued.
"""
import numpy as np
import pytest
import torch

import workloads as w
from oracle import admm as oadmm
from oracle import models as omodels
from oracle import qp as oqp

from test_gpu_parity import _compare, _run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_24039_gb300 import build
    build.build()


def _scaled_floor(pb, i, o):
    """FP32 residual floors (as tests/test_gpu_parity._fp32_floor) evaluated on the
    rescaled QP at the oracle's solution, in the scaled units the residuals of a
    rescaled solve are reported in."""
    inst = pb.instance(i)
    q = oqp.build_qp(inst, o["z"])
    sq, Dv, Ef, Eg = oadmm.rescale_qp(q, inst["scale"], omodels.selector_rows(inst))
    x = np.abs(o["z"].reshape(-1) / Dv)
    yf, yg = np.abs(o["yf"].reshape(-1) / Ef), np.abs(o["yg"].reshape(-1) / Eg)
    C, G, P = abs(sq["C"]).tocsr(), abs(sq["G"]).tocsr(), abs(sq["P"]).tocsc()
    prim = np.concatenate([C @ x + np.abs(sq["c"]), G @ x])
    m_prim = max(C.getnnz(axis=1).max(), G.getnnz(axis=1).max()) + 1
    dual = P @ x + np.abs(sq["q"]) + C.T @ yf + G.T @ yg
    m_dual = (P.getnnz(axis=0) + C.tocsc().getnnz(axis=0) + G.tocsc().getnnz(axis=0)).max() + 1
    u = 2.0 ** -24
    return u * np.sqrt(m_prim) * float(np.max(prim)), u * np.sqrt(m_dual) * float(np.max(dual))


def _di_batch(seed=11):
    pb = w.double_integrator(B=6, N=20, max_admm=200)
    pb.N[:] = [20, 1, 2, 7, 13, 19]
    for i in range(6):
        pb.Qd[i, int(pb.N[i]), :] = 10 * pb.Qd[i, 0, :]
    rng = np.random.default_rng(seed)
    pb.scale = np.exp(rng.uniform(np.log(0.3), np.log(5.0), size=(pb.B, pb.n)))   # units from 1/4 to 4
    return pb


@pytest.mark.parametrize("solver", [pytest.param(2, id="smem_cr"), pytest.param(3, id="global_cr"),
                                    pytest.param(4, id="warp_ldl")])
def test_rescaled_double_integrator(solver):
    pb = _di_batch()
    s, sol, _ = _run(pb, solver=solver)
    _compare(pb, sol, range(pb.B), sensitivity=True, floor=_scaled_floor)
    assert np.mean(oadmm.pow2_floor(pb.scale) != 1.0) > 0.5


@pytest.mark.parametrize("solver", [pytest.param(2, id="smem_cr"), pytest.param(4, id="warp_ldl")])
def test_rescaled_racing_equal_iterations(solver):
    pb = w.racing(B=8, N=50, max_sqp=1, max_admm=100)
    pb.scale = w.magnitude_scales(pb)
    s, sol, _ = _run(pb, solver=solver)
    _compare(pb, sol, range(8), sensitivity=True, floor=_scaled_floor)


def test_rescaled_model_mix():
    """Double integrator, bicycle and quadrotor (thrust bounds [0, 10] scaled by 8)
    in one batch, each model group on its shared-memory kernel."""
    pb = w.uneven(B=12, N_lo=10, N_hi=40, seed=77, max_sqp=1, max_admm=100)
    pb.scale = w.magnitude_scales(pb)
    s, sol, _ = _run(pb, solver=2)
    _compare(pb, sol, range(pb.B), sensitivity=True, floor=_scaled_floor)


def test_rescaled_forms_agree_bitwise():
    pb = w.racing(B=8, N=40, max_sqp=3, max_admm=30)
    pb.N[:] = [40, 7, 33, 1, 40, 20, 12, 39]
    pb.scale = w.magnitude_scales(pb)
    _, a, _ = _run(pb, solver=2)
    _, b, _ = _run(pb, solver=3)
    _, c, _ = _run(pb, solver=7)
    for k in ("z", "xi", "y_eq", "y_ineq", "status", "stats"):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(b[k], c[k]), k


def test_unit_scales_change_nothing():
    pb = w.racing(B=6, N=30, max_sqp=3, max_admm=30)
    _, a, _ = _run(pb, solver=2)
    pb.scale = np.ones((pb.B, pb.n))
    _, b, _ = _run(pb, solver=2)
    pb.scale[:, :] = 1.5           # rounds down to 1
    _, c, _ = _run(pb, solver=2)
    for k in ("z", "xi", "y_eq", "y_ineq", "status", "stats"):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a[k], c[k]), k


def test_rescaled_cluster_team_matches_single_cta():
    pb = w.double_integrator(B=2, N=700, max_admm=150)
    pb.N[:] = [700, 301]
    for i in range(2):
        pb.Qd[i, int(pb.N[i]), :] = 10 * pb.Qd[i, 0, :]
    pb.scale = np.tile(np.array([2.0, 2.0, 1.0, 1.0, 0.5, 0.5]), (2, 1))
    _, a, _ = _run(pb, solver=3)
    _, b, _ = _run(pb, solver=6)
    _compare(pb, a, range(2), sensitivity=True, floor=_scaled_floor)
    _compare(pb, b, range(2), sensitivity=True, floor=_scaled_floor)
    assert np.array_equal(a["status"], b["status"])


def test_host_entry_with_scales_equals_device_entry():
    from paper_2606_24039_gb300 import Solver, tensors_from_batch
    pb = w.racing(B=4, N=30, max_sqp=2, max_admm=30)
    pb.scale = w.magnitude_scales(pb)
    s = Solver.from_batch(pb, device="cuda", solver=2)
    dev = {k: v.cpu() for k, v in s.tmpc_solve(s.x0, z_init=s.z_init).items()}
    torch.cuda.synchronize()
    ht = {k: (None if v is None else v.cpu().pin_memory()) for k, v in tensors_from_batch(pb, "cuda").items()}
    out = {k: torch.zeros_like(v).pin_memory() for k, v in dev.items()}
    s.tmpc_solve_host(ht, ht["x0"], out, z_init_host=ht["z_init"])
    torch.cuda.synchronize()
    for k in ("z", "xi", "y_eq", "y_ineq", "status", "stats"):
        assert torch.equal(out[k], dev[k]), k
    s.close()


def test_scale_is_refused_on_the_generic_kernel():
    from paper_2606_24039_gb300 import Solver, TmpcError, options_from, tensors_from_batch, tmpc_solve_static
    pb = w.double_integrator(B=2, N=10, max_admm=20)
    pb.scale = np.full((pb.B, pb.n), 2.0)
    s = Solver.from_batch(pb, device="cuda", solver=1)
    with pytest.raises(TmpcError, match="generic kernel"):
        s.tmpc_solve(s.x0)
    s.close()
    tr = w.tracking(B=2, max_admm=20)
    tr.scale = np.full((tr.B, tr.n), 2.0)
    s = Solver.from_batch(tr, device="cuda")
    with pytest.raises(TmpcError, match="generic kernel"):
        s.tmpc_solve(s.x0)
    s.close()
    t = tensors_from_batch(pb, "cuda")
    dims = dict(batch=pb.B, N_max=pb.N_max, nx=pb.nx, nu=pb.nu, ng=pb.ng, n_dyn=pb.n_dyn, n_track=pb.n_track)
    out = {k: torch.zeros((pb.B,) + tuple(v.shape[1:]), device="cuda") for k, v in
           (("z", t["ref"]), ("xi", t["lo"]), ("y_eq", t["Qd"]), ("y_ineq", t["lo"]))}
    out["status"] = torch.zeros(pb.B, dtype=torch.int32, device="cuda")
    out["stats"] = None
    with pytest.raises(TmpcError, match="scale"):
        tmpc_solve_static(dims, t, t["x0"], out, options_from(pb.opts, solver=1))
