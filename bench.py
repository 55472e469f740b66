"""Throughput benchmark of the batched SQP/ADMM OCP solver on one node.

Default workload: kinematic-bicycle racing, B = 1024 instances, N = 50,
implicit midpoint dynamics, L1+L2-softened track constraint, control-rate
cost, 10 SQP x 50 ADMM iterations (FP32 on the GPU).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

One step = one forward solve of the whole batch (every instance, every SQP and
ADMM iteration); a second timed pass measures forward + backward.  Inputs are
resident in HBM; the L2 is flushed (a 512 MB write) between timed steps.  The
`e2e` figure times the host-memory entry point (tmpc_solve_host): copy of every
parameter array from pinned host memory, the solve, and the copy of the whole
solution back.  `--impl reference` times the FP64 CPU oracle (the baseline arm)
on a bounded sample of the same workload on the host cores.

Under torchrun (N > 1) every rank solves its own batch on its own GPU (weak
scaling, no collective on the data path); rank 0 prints one JSON line with the
max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "OCP solves/sec (fwd and fwd+bwd) at 1e-5 KKT residual; % of HBM/FP32 roofline"
UNIT = "solves/s"

# Algorithmic FP32 work of the path per stage, counted from the dense block
# operations of the method's formulas for a model with n = nx + nu, nx, ng;
# an FMA counts 2.  For the bicycle (8, 6, 5): 1056, 4992, 368 and 164.
def flop_admm_stage(n, nx, ng):
    # C'(.) and G'(.) of eta, block LDL' solve (6 n^2), C x~, G x~, relaxation, projection, duals
    return 8 * nx * n + 4 * ng * n + 6 * n * n + 3 * n + 9 * nx + 10 * ng


def flop_factor_stage(n, nx, ng):
    # rho_f (A+'A+ + A-'A-) and Phi_t (6 n^2 nx), rho_g G'G (2 n^2 ng), Schur update, pivot inverse, off-diagonal factor
    return 6 * n * n * nx + 2 * n * n * ng + 4 * n ** 3


def flop_lin_stage(n, nx, ng):
    return 6 * nx * n + 10 * n           # Jacobian products, cost gradient, shifted bounds


def flop_merit_stage(n, nx, ng):
    return 2 * nx * n + 6 * n + 4 * ng   # dynamics residual, cost, violation per line-search candidate


def bytes_admm_stage(n, nx, lti):
    # factor blocks (D^-1, off-diagonal factor) and, for time-varying models, A^-, A^+ read per iteration
    return 4 * (2 * n * n + (0 if lti else 2 * nx * n))


SMS, FP32_LANES = 152, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="racing",
                    choices=["racing", "double_integrator", "tracking", "uneven", "long_horizon"],
                    help="racing (default): bicycle B=1024 N=50; double_integrator: B=1 N=20; "
                         "tracking: linear nx=48 nu=20 N=32 B=512; uneven: B=4096 N in 10..200, "
                         "three models; long_horizon: bicycle B=8 N=8192")
    ap.add_argument("--batch", type=int, default=0, help="instances (0 = the workload's size)")
    ap.add_argument("--horizon", type=int, default=0, help="horizon N (0 = the workload's; fixed-N workloads)")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="oracle instances timed for cpu_baseline (0 = about 10-30 CPU-seconds of the workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-bwd", action="store_true", help="time the forward pass only")
    ap.add_argument("--solver", type=int, default=0, help="0 auto, 1 generic sequential LDL', 2 shared-memory CR, 3 CR on global arenas, "
                    "4 warp-sequential LDL', 5 warp LDL' on global arenas")
    ap.add_argument("--skip-e2e", action="store_true", help="skip the host-memory end-to-end timing")
    ap.add_argument("--threads", type=int, default=0, help="threads per instance (0 = library default)")
    ap.add_argument("--clocks-csv", default=None,
                    help="also keep the raw nvidia-smi clock samples of the timed region in this CSV file")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the launch form chosen at setup (default: tmpc_autotune picks it per model group)")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain per-phase form (one launch per phase, eager and as a CUDA graph)")
    return ap.parse_args()


CPU_SAMPLE = {"racing": 128, "double_integrator": 512, "tracking": 96, "uneven": 192, "long_horizon": 16}

WORKLOADS = {
    # name: (generator, default batch, default horizon, seed, description)
    "racing": ("racing", 1024, 50, 1002, "kinematic-bicycle racing (implicit midpoint, L1+L2 soft track row, "
                                         "rate cost, progress cost)"),
    "double_integrator": ("double_integrator", 1, 20, 1001, "2-D double integrator, box bounds on u and v"),
    "tracking": ("tracking", 512, 32, 1003, "linear tracking nx=48 nu=20, MLP cost weights, |u| <= 1"),
    "uneven": ("uneven", 4096, 0, 1004, "uneven batch N in 10..200, double integrator / bicycle / quadrotor 1:2:1"),
    "long_horizon": ("long_horizon", 8, 8192, 1005, "kinematic-bicycle racing, dt=0.01, closed 2 km track"),
}


def make_batch(name, B, N, seed):
    import workloads as w
    gen = getattr(w, WORKLOADS[name][0])
    if name == "uneven":
        return gen(B=B, seed=seed)
    return gen(B=B, N=N, seed=seed)


def workload(args, rank=0):
    _, B0, N0, seed, _ = WORKLOADS[args.workload]
    return make_batch(args.workload, args.batch or B0, args.horizon or N0, seed + 7919 * rank)


def config_of(args, pb):
    desc = WORKLOADS[args.workload][4]
    Ns = f"N={pb.N_max}" if np.all(pb.N == pb.N_max) else f"N={int(pb.N.min())}..{int(pb.N.max())}"
    return {"workload": f"{args.workload}: {desc}, B={pb.B} {Ns}, {pb.opts.max_sqp} SQP x {pb.opts.max_admm} ADMM",
            "batch": pb.B, "horizon": pb.N_max, "nx": pb.nx, "nu": pb.nu, "ng": pb.ng,
            "sqp_iters": pb.opts.max_sqp, "admm_iters": pb.opts.max_admm,
            "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{args.gpus}",
            "solver": {0: "auto", 1: "generic sequential block LDL'", 2: "shared-memory block cyclic reduction",
                       3: "block cyclic reduction, global-memory arenas",
                       4: "shared-memory sequential block LDL' by one warp",
                       5: "sequential block LDL' by one warp, global-memory arenas"}[args.solver]}


# ----------------------------------------------------------------------------
# CPU oracle timing (baseline / reference arm)
# ----------------------------------------------------------------------------
_WORKER_BATCH = None


def _init_worker(name, B, N, seed):
    global _WORKER_BATCH
    _WORKER_BATCH = make_batch(name, B, N, seed)


def _oracle_one(i):
    from oracle import sqp
    pb = _WORKER_BATCH
    inst = pb.instance(i % pb.B)
    t = time.perf_counter()
    sqp.solve(inst, pb.opts)
    return time.perf_counter() - t


def oracle_rate(args, n_inst, cores):
    """Solve n_inst instances of the workload with the FP64 oracle on `cores`
    processes; returns (solves/s, wall seconds, summed CPU seconds).  Instance
    generation happens once per worker, before the timed map."""
    # one single-threaded process per core: the BLAS/LAPACK calls of the oracle must not
    # start their own thread pools (the spawned workers read these at numpy import)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    _, B0, N0, seed, _ = WORKLOADS[args.workload]
    with ctx.Pool(cores, initializer=_init_worker,
                  initargs=(args.workload, min(n_inst, args.batch or B0), args.horizon or N0, seed)) as pool:
        pool.map(_oracle_one, range(cores), chunksize=1)   # imports, warm caches
        t = time.perf_counter()
        times = pool.map(_oracle_one, range(n_inst), chunksize=1)
        wall = time.perf_counter() - t
    return n_inst / wall, wall, float(np.sum(times))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    per_step = max(cores, min(args.cpu_sample or CPU_SAMPLE[args.workload], 4 * cores))
    for _ in range(max(args.warmup, 0) and 1):
        oracle_rate(args, cores, cores)
    vals, walls = [], []
    for _ in range(args.steps):
        v, wall, _ = oracle_rate(args, per_step, cores)
        vals.append(v)
        walls.append(wall)
    value = float(np.median(vals))
    pb = workload(args)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.median(walls)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args, pb),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} instances of the workload per step, FP64 numpy/scipy oracle, "
                                       f"one process per core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, gpu_index, path=None):
        import tempfile
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to `path` when given (--clocks-csv), else to a temporary file
        self.path = path or os.path.join(tempfile.gettempdir(), f"tmpc_clocks_{os.getpid()}_gpu{gpu_index}.csv")

    def __enter__(self):
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap,timestamp", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(1.0)   # let the sampler start before the timed region
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, t0=None, t1=None):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return None
        if t0 is not None:
            import datetime
            keep = []
            for r in rows:
                try:
                    ts = datetime.datetime.strptime(r[-1].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except Exception:
                    continue
                if t0 <= ts <= t1:
                    keep.append(r)
            rows = keep or rows
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def _model_dims(pb):
    import workloads as w
    dims = np.array([w.model_dims(int(m), pb.nx, pb.nu, pb.ng) for m in pb.model], dtype=np.float64)
    return dims[:, 0] + dims[:, 1], dims[:, 0], dims[:, 2]


def algorithmic_flops(pb, stats):
    """FP32 flops the method needs for the solves just run (counts from the stats)."""
    n, nx, ng = _model_dims(pb)
    T = pb.N.astype(np.float64) + 1.0
    admm = stats[:, 1].astype(np.float64)
    fact = stats[:, 5].astype(np.float64)
    sqp = stats[:, 0].astype(np.float64)
    n_ls = float(pb.opts.n_ls) if pb.opts.n_ls > 1 else 0.0
    return float(np.sum(T * (admm * flop_admm_stage(n, nx, ng) + fact * flop_factor_stage(n, nx, ng)
                             + (sqp + 1) * flop_lin_stage(n, nx, ng) + sqp * n_ls * flop_merit_stage(n, nx, ng))))


def algorithmic_bytes(pb, stats):
    """Bytes the ADMM iterations must stream when the factors live in HBM (the
    generic kernel's workspace): factor blocks and time-varying Jacobians."""
    import workloads as w
    n, nx, ng = _model_dims(pb)
    lti = np.isin(pb.model, (w.MODEL_DI, w.MODEL_LINEAR))
    T = pb.N.astype(np.float64) + 1.0
    admm = stats[:, 1].astype(np.float64)
    per = np.where(lti, 4 * 2 * n * n, 4 * (2 * n * n + 2 * nx * n))
    return float(np.sum(T * admm * per))


FAST_MODELS = (0, 2, 3)   # models with a compile-time-sized shared-memory kernel


def n_launch_groups(pb, solver):
    """Solve kernels one forward call launches: one per fast-model group present,
    plus one generic launch for every other model (all models when solver = 1)."""
    models = set(int(m) for m in np.unique(pb.model))
    if solver == 1:
        return 1
    fast = len(models & set(FAST_MODELS))
    return fast + (1 if models - set(FAST_MODELS) else 0)


KERNEL_SOURCES = ("tmpc_fast_kernels.cuh", "tmpc_fast_model.cuh", "tmpc_fast_bicycle.cu", "tmpc_fast.cuh", "tmpc_fast_api.h",
                  "tmpc_solver.cuh", "tmpc_models.cuh", "tmpc_backward.cuh")


def sources_digest():
    """SHA-256 over the sources of the shared-memory solve kernel's translation unit."""
    import hashlib
    d = os.path.join(ROOT, "paper_2606_24039_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def measured_peak(key, fallback):
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key])
    except Exception:
        return fallback


FORM_NAMES = {2: "fast::solve_kernel<{m}, kCR>", 3: "fast::solve_kernel<{m}, kCR> (global arenas)",
              4: "fast::solve_kernel<{m}, kLDL>", 5: "fast::solve_kernel<{m}, kLDL> (global arenas)",
              6: "fast::solve_kernel_cluster<{m}, kCR>", 7: "fast::plain_* <{m}> (per-phase form)"}


def kernel_name(pb, solver, forms=None):
    """The solve kernel(s) of one forward call; forms maps a model id to the launch
    form the autotuner kept (tmpc_tune_result.solver)."""
    import workloads as w
    names = {w.MODEL_DI: "MODEL_DI", w.MODEL_BICYCLE: "MODEL_BICYCLE", w.MODEL_QUAD: "MODEL_QUAD"}
    ks = []
    for m in sorted(set(int(v) for v in np.unique(pb.model))):
        if m not in names or solver == 1:
            ks.append("solve_kernel (generic)")
            continue
        f = (forms or {}).get(m, solver if solver >= 2 else 2)
        ks.append(FORM_NAMES[f].format(m=names[m]))
    return " + ".join(sorted(set(ks)))


def launches_per_step(pb, solver, forms=None):
    """Kernels launched by one forward call and by one backward call: per fast-model
    group one persistent launch (the plain form: one per phase), one generic launch
    for the other models; backward: one per cyclic-reduction group plus one generic
    launch for the rest."""
    models = set(int(m) for m in np.unique(pb.model))
    if solver == 1:
        return 1, 1
    if not forms:
        forms = {m: (solver if solver >= 2 else 2) for m in models & set(FAST_MODELS)}
    other = bool(models - set(forms))
    fwd = sum(2 + pb.opts.max_sqp * (2 + pb.opts.max_admm) if f == 7 else 1 for f in forms.values()) + int(other)
    bwd = sum(1 for f in forms.values() if f not in (4, 5)) + int(other or any(f in (4, 5) for f in forms.values()))
    return fwd, bwd


def measured_traffic(args, pb):
    """DRAM bytes (read + write) per launch of the solve kernel from the committed
    ncu summary, scaled to this batch by instances; None when the kernel sources
    changed since the counters were taken or no summary matches the workload."""
    path = os.path.join(ROOT, "profiles", "solve_kernel_bicycle_racing_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    if (rec.get("sources_sha256") != sources_digest() or rec.get("horizon") != pb.N_max
            or rec.get("workload_name", "racing") != args.workload):
        return None
    return rec["dram_bytes_per_launch"] * pb.B / rec["batch"]


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        n = max(cores, args.cpu_sample or CPU_SAMPLE[args.workload])
        v, wall, cpu_s = oracle_rate(args, n, cores)
        cpu_base = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                    "sample": f"{n} instances of the same workload (FP64 numpy/scipy oracle, one process per core, "
                              f"{cpu_s:.1f} s CPU)"}
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2606_24039_gb300 import Solver, build, tensors_from_batch
    build.build()
    pb = workload(args, rank)
    s = Solver.from_batch(pb, device="cuda", solver=args.solver, threads=args.threads)
    sol = s.alloc_solution("cuda")
    warm = s.z_init is not None
    tune, forms = None, None
    if args.solver == 0 and not args.no_autotune:
        # the autotuner times each launch form of every model group on this batch
        # (whole solves from the same initial guess as the timed steps)
        if warm:
            sol["z"].copy_(s.z_init)
            for k in ("xi", "y_eq", "y_ineq"):
                sol[k].zero_()
        tune = s.tmpc_autotune(s.x0, init=sol if warm else None, reps=2, trial_sqp=0)
        forms = {r["model"]: r["solver"] for r in tune if r["model"] >= 0}
    dLdz = torch.randn((pb.B, pb.N_max + 1, pb.n), device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    ev = lambda: torch.cuda.Event(enable_timing=True)

    def restart():
        # every step starts from the same initial guess (zero slacks and multipliers)
        if warm:
            sol["z"].copy_(s.z_init)
            for k in ("xi", "y_eq", "y_ineq"):
                sol[k].zero_()

    def step(kev=None):
        restart()
        if kev is not None:
            kev[0].record(stream)
        s.tmpc_solve(s.x0, sol, warm_start=warm)
        if kev is not None:
            kev[1].record(stream)

    def step_fb(kev=None):
        step(kev)
        s.tmpc_backward(s.x0, sol, dLdz)

    for _ in range(args.warmup):
        step()
        if not args.skip_bwd:
            step_fb()
    torch.cuda.synchronize()

    def timed(fn):
        times, ktimes = [], []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            a, b, kev = ev(), ev(), (ev(), ev())
            a.record(stream)
            fn(kev)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            ktimes.append(kev[0].elapsed_time(kev[1]))
        return times, ktimes

    with Clocks(local, args.clocks_csv) as clk:
        t0 = time.time()
        t_fwd, k_fwd = timed(step)
        t_fb, _ = timed(step_fb) if not args.skip_bwd else ([float("nan")], None)
        t1 = time.time()
    clocks = clk.summary(t0, t1)
    stats = sol["stats"].cpu().numpy()
    status = sol["status"].cpu().numpy()
    kkt = stats[:, 6]
    l_fwd, l_bwd = launches_per_step(pb, args.solver, forms)
    launches = args.steps * l_fwd + (0 if args.skip_bwd else args.steps * (l_fwd + l_bwd))

    # the plain per-phase form of the same solve: one launch per phase, eager and
    # captured as a CUDA graph (the baseline the persistent kernel is compared with)
    plain = None
    if not args.no_plain and args.workload in ("racing", "double_integrator", "uneven") and args.solver in (0, 2):
        sp = Solver.from_batch(pb, device="cuda", solver=7, threads=args.threads)
        solp = sp.alloc_solution("cuda")
        side = torch.cuda.Stream()

        def pstep():
            if warm:
                solp["z"].copy_(sp.z_init)
                for k in ("xi", "y_eq", "y_ineq"):
                    solp[k].zero_()
            sp.tmpc_solve(sp.x0, solp, warm_start=warm)

        for _ in range(2):
            pstep()
        torch.cuda.synchronize()
        n_plain = max(2, min(args.steps, 5))

        def time_fn(fn):
            ts = []
            for _ in range(n_plain):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                a, b = ev(), ev()
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            return float(np.mean(ts))

        eager_ms = time_fn(pstep)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            pstep()
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=side):
                pstep()
        torch.cuda.synchronize()
        graph_ms = time_fn(g.replay)
        kp = solp["stats"][:, 6].cpu().numpy()
        groups_p = n_launch_groups(pb, 2)
        plain = {"eager_ms": eager_ms, "graph_ms": graph_ms, "persistent_ms": float(np.mean(t_fwd)),
                 "launches_per_step": groups_p * (2 + pb.opts.max_sqp * (2 + pb.opts.max_admm)),
                 "kkt_median": float(np.median(kp)), "kkt_median_persistent": float(np.median(kkt)),
                 "speedup_vs_eager": eager_ms / float(np.mean(t_fwd)), "speedup_vs_graph": graph_ms / float(np.mean(t_fwd))}
        del g
        sp.close()

    # end to end through the host-memory entry point
    hp = {k: (v.cpu().pin_memory() if v is not None else None) for k, v in tensors_from_batch(pb, "cpu").items()}
    ho = {k: v.cpu().pin_memory() for k, v in s.alloc_solution("cpu").items()}
    h2d = sum(v.numel() * v.element_size() for v in hp.values() if v is not None)
    d2h = sum(v.numel() * v.element_size() for v in ho.values())
    for _ in range(0 if args.skip_e2e else max(1, args.warmup)):
        s.tmpc_solve_host(hp, hp["x0"], ho, z_init_host=hp["z_init"])
    e2e_t = [float("nan")]
    for _ in range(0 if args.skip_e2e else args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        s.tmpc_solve_host(hp, hp["x0"], ho, z_init_host=hp["z_init"])
        e2e_t.append(time.perf_counter() - t)
    e2e_t = [v for v in e2e_t if v == v] or [float("nan")]

    ms_f = float(np.mean(t_fwd))
    ms_fb = float(np.mean(t_fb))
    ms_e2e = 1e3 * float(np.mean(e2e_t))
    if world > 1:   # the slowest rank sets the job time (no collective on the data path)
        from paper_2606_24039_gb300.shard import max_over_ranks
        ms_f, ms_fb, ms_e2e = (max_over_ranks(v, device="cuda") for v in (ms_f, ms_fb, ms_e2e))
    total = pb.B * world
    value = total / (ms_f * 1e-3)
    flops = algorithmic_flops(pb, stats)
    ms_k = float(np.mean(k_fwd))          # the solve kernel(s) of one forward step, on the launching stream
    peak_clock = 2070.0
    fp32_peak = SMS * FP32_LANES * 2 * peak_clock * 1e6 / 1e12
    if args.workload == "tracking":
        # factors of 0.74 MB per instance do not fit on chip: streamed from HBM every ADMM iteration
        achieved = algorithmic_bytes(pb, stats) / (ms_k * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": measured_peak("hbm_gbs", 6800.0), "unit": "GB/s",
                "flops_tflops": flops / (ms_k * 1e-3) / 1e12,
                "peak_note": "STREAM-style copy bandwidth of this GPU pool (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        achieved = flops / (ms_k * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "peak_note": "FP32 FMA peak = 152 SM x 128 lanes x 2 flop x 2070 MHz (derived)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = measured_traffic(args, pb)
    roof["kernel"] = kernel_name(pb, args.solver, forms)
    roof["kernel_ms"] = ms_k
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_f, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_of(args, pb),
            "fwd_bwd": {"value": total / (ms_fb * 1e-3), "unit": UNIT, "ms_per_step": ms_fb},
            "clocks": clocks,
            "e2e": {"value": total / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu_base,
            "plain_form": plain,
            "autotune": tune,
            "quality": {"kkt_median": float(np.median(kkt)), "kkt_p90": float(np.percentile(kkt, 90)),
                        "frac_kkt_le_1e-5": float(np.mean(kkt <= 1e-5)),
                        "status_counts": {str(k): int(v) for k, v in zip(*np.unique(status, return_counts=True))},
                        "admm_iters_mean": float(stats[:, 1].mean()), "factorizations_mean": float(stats[:, 5].mean())},
        }
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
