"""Throughput benchmark of the batched SQP/ADMM OCP solver on one node.

Headline workload (the largest single-GPU configuration): the uneven batch,
4096 instances whose horizons are drawn from 10..200 and whose models mix
the double integrator, the kinematic bicycle (implicit midpoint, soft track
row) and the planar quadrotor 1:2:1, 10 SQP x 50 ADMM iterations, forward
and forward + backward in one persistent launch per model group (FP32; the
direct backward of the small models in FP64).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload uneven|racing|tracking|long_horizon|double_integrator|linear_rl] [--no-suite]

One step = one forward solve of the whole batch (every instance, every SQP
and ADMM iteration); a second timed pass measures forward + backward.  Inputs
are resident in HBM; the L2 is flushed (a 512 MB write) between timed steps.
`e2e` times the host-memory entry point (tmpc_solve_host): the copy of every
parameter array from pinned host memory, the solve, and the copy of the whole
solution back.  With the default workload the line also carries
  - `workloads`: the racing (B=1024, N=50), tracking (B=512, nx=48, nu=20,
    N=32), long-horizon (B=8, N=8192), double-integrator (B=1, N=20) and
    linear-system RL (B=64, N=40, nx=8, nu=4, tolerance 1e-5) workloads,
    each timed the same way (fewer steps) with its dominant kernel's roofline;
  - `at_1e-5`: every workload solved to the tolerance 1e-5 (early exit at
    eps_abs = eps_rel = eps_c = 1e-5, at most 1000 ADMM iterations per QP,
    at most 10 SQP iterations for the linear problems and 20 otherwise):
    solves/s and the fraction of instances whose SQP KKT residual
    (Eq. sqp_stop) reaches 1e-5.
`--impl reference` times the FP64 CPU oracle (the baseline arm) on a bounded
sample of the same workload on the host cores.

Under torchrun (N > 1) every rank solves its longest-processing-time-first shard
of a job batch N times the one-GPU batch on its own GPU (weak scaling, no
collective on the data path); rank 0 prints one JSON line with the
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




FP32_LANES_PER_SM = 128   # FP32 FMA lanes per Blackwell SM


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="uneven", choices=list(WORKLOADS),
                    help="uneven (default): B=4096 N in 10..200, three models; racing: bicycle B=1024 N=50; "
                         "tracking: linear nx=48 nu=20 N=32 B=512; long_horizon: bicycle B=8 N=8192; "
                         "double_integrator: B=1 N=20; linear_rl: B=64 N=40 nx=8 nu=4 at tolerance 1e-5")
    ap.add_argument("--batch", type=int, default=0, help="instances (0 = the workload's size)")
    ap.add_argument("--horizon", type=int, default=0, help="horizon N (0 = the workload's; fixed-N workloads)")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="oracle instances timed for cpu_baseline (0 = about 10-30 CPU-seconds of the workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-bwd", action="store_true", help="time the forward pass only")
    ap.add_argument("--solver", type=int, default=0, help="0 auto, 1 generic sequential LDL', 2 shared-memory CR, "
                    "3 CR on global arenas, 4 warp-sequential LDL', 5 warp LDL' on global arenas, 6 cluster CR")
    ap.add_argument("--skip-e2e", action="store_true", help="skip the host-memory end-to-end timing")
    ap.add_argument("--threads", type=int, default=0, help="threads per instance (0 = library default)")
    ap.add_argument("--clocks-csv", default=None,
                    help="also keep the raw nvidia-smi clock samples of the timed region in this CSV file")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the launch form chosen at setup (default: tmpc_autotune picks it per model group)")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain per-phase form (one launch per phase, eager and as a CUDA graph)")
    ap.add_argument("--no-suite", action="store_true",
                    help="only the selected workload: no `workloads` and no `at_1e-5` records")
    return ap.parse_args()


CPU_SAMPLE = {"racing": 128, "double_integrator": 512, "tracking": 96, "uneven": 160, "long_horizon": 16,
              "linear_rl": 256, "humanoid": 256}

WORKLOADS = {
    # name: (generator, default batch, default horizon, seed, description)
    "uneven": ("uneven", 4096, 0, 1004, "uneven batch N in 10..200, double integrator / bicycle / quadrotor 1:2:1"),
    "racing": ("racing", 1024, 50, 1002, "kinematic-bicycle racing (implicit midpoint, L1+L2 soft track row, "
                                         "rate cost, progress cost)"),
    "tracking": ("tracking", 512, 32, 1003, "linear tracking nx=48 nu=20, MLP cost weights, |u| <= 1"),
    "long_horizon": ("long_horizon", 8, 8192, 1005, "kinematic-bicycle racing, dt=0.01, closed 2 km track"),
    "double_integrator": ("double_integrator", 1, 20, 1001, "2-D double integrator, box bounds on u and v"),
    "linear_rl": ("linear_rl", 64, 40, 1006, "linear-system RL: x+ = A x + B u + b, nx=8 nu=4, |u| <= 1, "
                                             "Q = diag(theta), tolerance 1e-5 (<= 1000 ADMM per QP)"),
    "humanoid": ("humanoid", 100, 20, 1007, "single-rigid-body humanoid balance, nx=12 nu=6, RK4 dt=0.025, "
                                           "Q = diag(exp(theta)), box on the foot forces"),
}
SUITE = ("racing", "tracking", "long_horizon", "double_integrator", "linear_rl", "humanoid")
LINEAR = ("tracking", "double_integrator", "linear_rl")


def make_batch(name, B, N, seed, **kw):
    import workloads as w
    gen = getattr(w, WORKLOADS[name][0])
    if name == "uneven":
        return gen(B=B, seed=seed, **kw)
    return gen(B=B, N=N, seed=seed, **kw)


def workload(args, rank=0, name=None, world=1):
    """The workload's batch for this rank.  Under torchrun (world > 1) the job's
    batch is world times the one-GPU batch, drawn once with the same seed on every
    rank, and each rank takes its longest-processing-time-first shard of it (work
    (N+1) n^2 per instance): the per-GPU work stays that of the one-GPU run (weak
    scaling), balanced across ranks."""
    import workloads as w
    name = name or args.workload
    _, B0, N0, seed, _ = WORKLOADS[name]
    B = (args.batch if name == args.workload else 0) or B0
    N = (args.horizon if name == args.workload else 0) or N0
    if world <= 1:
        return make_batch(name, B, N, seed)
    from paper_2606_24039_gb300.shard import instance_work, shard_of
    full = make_batch(name, B * world, N, seed)
    n = np.array([sum(w.model_dims(int(m), full.nx, full.nu, full.ng)[:2]) for m in full.model])
    return full.subset(shard_of(instance_work(full.N, n), world, rank))


def describe(name, pb, world=1, solver=0):
    desc = WORKLOADS[name][4]
    Ns = f"N={pb.N_max}" if np.all(pb.N == pb.N_max) else f"N={int(pb.N.min())}..{int(pb.N.max())}"
    its = (f"{pb.opts.max_sqp} SQP x {pb.opts.max_admm} ADMM" if not pb.opts.early_exit else
           f"to tolerance {pb.opts.eps_c:g} (<= {pb.opts.max_sqp} SQP, <= {pb.opts.max_admm} ADMM per QP)")
    return {"workload": f"{name}: {desc}, B={pb.B} {Ns}, {its}",
            "batch": pb.B, "horizon": pb.N_max, "nx": pb.nx, "nu": pb.nu, "ng": pb.ng,
            "sqp_iters": pb.opts.max_sqp, "admm_iters": pb.opts.max_admm, "early_exit": bool(pb.opts.early_exit),
            "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{world}",
            "solver": {0: "auto", 1: "generic sequential block LDL'", 2: "shared-memory block cyclic reduction",
                       3: "block cyclic reduction, global-memory arenas",
                       4: "shared-memory sequential block LDL' by one warp",
                       5: "sequential block LDL' by one warp, global-memory arenas",
                       6: "block cyclic reduction by one thread-block cluster per instance"}.get(solver, str(solver))}


def config_of(args, pb):
    return describe(args.workload, pb, args.gpus, args.solver)


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
    for the other models; backward: per cyclic-reduction CTA group three (the
    backward pass, the kernel of the direct solve's sweeps, the finishing pass),
    per cluster group one, plus one generic launch for the rest."""
    models = set(int(m) for m in np.unique(pb.model))
    if solver == 1:
        return 1, 1
    if not forms:
        forms = {m: (solver if solver >= 2 else 2) for m in models & set(FAST_MODELS)}
    other = bool(models - set(forms))
    fwd = sum(2 + pb.opts.max_sqp * (2 + pb.opts.max_admm) if f == 7 else 1 for f in forms.values()) + int(other)
    bwd = sum(1 if f == 6 else 3 for f in forms.values() if f not in (4, 5)) + \
        int(other or any(f in (4, 5) for f in forms.values()))
    return fwd, bwd


def measured_traffic(name, pb, kernel):
    """DRAM bytes (read + write) per launch of a solve kernel from the committed
    ncu records, scaled to this batch by instances; None when the kernel sources
    changed since the counters were taken or no record matches."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*_traffic.json"))):
        try:
            rec = json.load(open(path))
        except Exception:
            continue
        if (rec.get("sources_sha256") == sources_digest() and rec.get("workload_name") == name
                and rec.get("kernel") == kernel and rec.get("horizon") == pb.N_max):
            return rec["dram_bytes_per_launch"] * pb.B / rec["batch"]
    return None


def max_sm_clock_mhz(gpu_index):
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        return float(out.stdout.strip().splitlines()[0])
    except Exception:
        return measured_peak("sm_max_mhz", 2070.0)


def fp32_peak(gpu_index):
    """FP32 FMA peak of the device: SM count (device properties) x 128 lanes x
    2 flop x the maximum SM clock (nvidia-smi); TFLOP/s, SMs, MHz."""
    import torch
    sms = torch.cuda.get_device_properties(gpu_index).multi_processor_count
    mhz = max_sm_clock_mhz(gpu_index)
    return sms * FP32_LANES_PER_SM * 2.0 * mhz * 1e6 / 1e12, sms, mhz


def fp32_probe():
    """FP32 FMA throughput measured by the library's probe (eight independent FMA
    chains per thread on every SM); TFLOP/s, or None if the probe failed."""
    import ctypes
    from paper_2606_24039_gb300 import _abi
    t, ms = ctypes.c_float(0.0), ctypes.c_float(0.0)
    code = _abi.load().tmpc_fp32_fma_probe(ctypes.byref(t), ctypes.byref(ms))
    return float(t.value) if code == 0 else None


GROUP_MODELS = {0: "MODEL_DI", 2: "MODEL_BICYCLE", 3: "MODEL_QUAD"}


def group_kernel(model, form):
    if model < 0 or form == 1:
        return "solve_kernel (generic)"
    return FORM_NAMES[form].format(m=GROUP_MODELS[model])


def group_members(pb, model, solver):
    """Instances of the model group `model` (-1: the generic kernel's group)."""
    m = np.asarray(pb.model)
    if solver == 1:
        return np.arange(pb.B)
    if model < 0:
        return np.flatnonzero(~np.isin(m, FAST_MODELS))
    return np.flatnonzero(m == model)


def roofline_of(name, pb, stats, gtimes, solver, peak):
    """Roofline of the forward kernel: the one persistent launch of a single
    model group, or, when the model groups run concurrently on their streams,
    their concurrent launches together (all their instances' work over the span
    of the longest launch); device times by CUDA events on the launching streams."""
    import workloads as w
    groups = [g for g in gtimes if g["fwd_ms"] > 0]
    if not groups:
        return None
    g = max(groups, key=lambda r: r["fwd_ms"])
    ms = g["fwd_ms"]
    if len(groups) > 1:
        idx = np.concatenate([group_members(pb, r["model"], solver) for r in groups])
        kernel = " + ".join(group_kernel(r["model"], r["form"]) for r in groups) + " (concurrent)"
        for r in groups:   # each group's own rate, for reference
            gi = group_members(pb, r["model"], solver)
            r["fwd_tflops"] = algorithmic_flops(pb.subset(gi), stats[gi]) / (r["fwd_ms"] * 1e-3) / 1e12
    else:
        idx = group_members(pb, g["model"], solver)
        kernel = group_kernel(g["model"], g["form"])
    sub = pb.subset(idx)
    st = stats[idx]
    lti = bool(np.all(np.isin(sub.model, (w.MODEL_LINEAR,))))
    if lti and g["model"] < 0:
        # factor blocks that do not fit on chip stream from HBM every ADMM iteration
        achieved = algorithmic_bytes(sub, st) / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": measured_peak("hbm_gbs", 6800.0), "unit": "GB/s",
                "peak_note": "STREAM-style copy bandwidth of this GPU pool (MEASURED_PEAKS.json hbm_gbs), of measured",
                "flops_tflops": algorithmic_flops(sub, st) / (ms * 1e-3) / 1e12}
    else:
        achieved = algorithmic_flops(sub, st) / (ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak[0], "unit": "TFLOP/s",
                "peak_note": f"FP32 FMA peak = {peak[1]} SMs (device properties) x {FP32_LANES_PER_SM} lanes x 2 flop "
                             f"x {peak[2]:.0f} MHz (maximum SM clock), derived"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = measured_traffic(name, pb, kernel)
    roof["kernel"] = kernel
    roof["kernel_ms"] = ms
    roof["instances"] = int(len(idx))
    return roof


def mean_group_times(samples):
    """Average the per-group device times of several steps (tmpc_group_times)."""
    out = []
    for k in range(len(samples[0])):
        rows = [s[k] for s in samples if k < len(s)]
        r = dict(rows[0])
        for f in ("fwd_ms", "bwd_ms"):
            vals = [x[f] for x in rows if x[f] > 0]
            r[f] = float(np.mean(vals)) if vals else -1.0
        out.append(r)
    return out


BACKENDS = {2: "direct", 0: "hybrid", 1: "refinement", 3: "adjoint_qp"}


def backward_backends(s, pb, sol, dLdz, flush, steps):
    """The backward solvers on the same forward solution: time of one tmpc_backward
    call (CUDA events, L2 flushed before each) and the relative deviation of each
    backend's gradients (x0, Q, R, ref) from the direct solve's."""
    import torch
    from paper_2606_24039_gb300 import options_from
    stream = torch.cuda.current_stream()
    keep = s.options
    out, ref = {}, None
    for b, label in BACKENDS.items():
        s.tmpc_set_options(options_from(keep, bwd_solver=b))
        g = s.tmpc_backward(s.x0, sol, dLdz)
        times = []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g = s.tmpc_backward(s.x0, sol, dLdz)
            e.record(stream)
            e.synchronize()
            times.append(a.elapsed_time(e))
        vec = torch.cat([g[k].reshape(pb.B, -1) for k in ("x0", "Qd", "Rd", "ref")], dim=1).double()
        if ref is None:
            ref = vec
        dev = ((vec - ref).norm(dim=1) / ref.norm(dim=1).clamp_min(1e-12)).cpu().numpy()
        fin = lambda v: float(v) if np.isfinite(v) else None
        out[label] = {"ms": float(np.mean(times)), "grad_dev_median": fin(np.median(dev)),
                      "grad_dev_p99": fin(np.percentile(dev, 99)), "nonfinite": int(np.sum(~np.isfinite(dev)))}
    s.tmpc_set_options(keep)
    return out


def measure(name, pb, args, peak, flush, steps, warmup, autotune=False, plain=False, e2e=False, bwd=True,
            solver=0, world=1, backends=False):
    """Time one workload: forward steps and forward + backward steps (CUDA events
    on the caller's stream, L2 flushed before each), the per-group kernel times
    (events on the launching streams), quality of the returned points; with
    backends, the backward solvers compared on the last forward solution."""
    import torch
    from paper_2606_24039_gb300 import Solver, tensors_from_batch
    s = Solver.from_batch(pb, device="cuda", solver=solver, threads=args.threads)
    sol = s.alloc_solution("cuda")
    warm = s.z_init is not None
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    rec = {"config": describe(name, pb, world, solver)}
    tune, forms = None, None
    if autotune and solver == 0:
        if warm:
            sol["z"].copy_(s.z_init)
            for k in ("xi", "y_eq", "y_ineq"):
                sol[k].zero_()
        tune = s.tmpc_autotune(s.x0, init=sol if warm else None, reps=2, trial_sqp=0)
        forms = {r["model"]: r["solver"] for r in tune if r["model"] >= 0}
        rec["autotune"] = tune
    dLdz = torch.randn((pb.B, pb.N_max + 1, pb.n), device="cuda")

    def restart():
        if warm:   # every step starts from the same initial guess (zero slacks and multipliers)
            sol["z"].copy_(s.z_init)
            for k in ("xi", "y_eq", "y_ineq"):
                sol[k].zero_()

    def step():
        restart()
        s.tmpc_solve(s.x0, sol, warm_start=warm)

    def step_fb():
        step()
        s.tmpc_backward(s.x0, sol, dLdz)

    for _ in range(warmup):
        step()
        if bwd:
            step_fb()
    torch.cuda.synchronize()

    def timed(fn):
        times, gts = [], []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            a, b = ev(), ev()
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            gts.append(s.tmpc_group_times())
        return times, gts

    t_fwd, g_fwd = timed(step)
    stats = sol["stats"].cpu().numpy()
    status = sol["status"].cpu().numpy()
    t_fb, g_fb = timed(step_fb) if bwd else ([float("nan")], None)
    gt = mean_group_times(g_fwd)
    if g_fb:
        gb = mean_group_times(g_fb)
        for r, q in zip(gt, gb):
            r["bwd_ms"] = q["bwd_ms"]
        gt += gb[len(gt):]
    kkt = stats[:, 6]
    l_fwd, l_bwd = launches_per_step(pb, solver, forms)
    ms_f, ms_fb = float(np.mean(t_fwd)), float(np.mean(t_fb))
    rec.update({
        "ms_per_step": ms_f, "value": pb.B / (ms_f * 1e-3), "unit": UNIT,
        "fwd_bwd": {"value": pb.B / (ms_fb * 1e-3), "unit": UNIT, "ms_per_step": ms_fb} if bwd else None,
        "group_times": gt,
        "roofline": roofline_of(name, pb, stats, gt, solver, peak),
        "gpu_launches": steps * l_fwd + (steps * (l_fwd + l_bwd) if bwd else 0),
        "quality": {"kkt_median": float(np.median(kkt)), "kkt_p90": float(np.percentile(kkt, 90)),
                    "frac_kkt_le_1e-5": float(np.mean(kkt <= 1e-5)),
                    "status_counts": {str(k): int(v) for k, v in zip(*np.unique(status, return_counts=True))},
                    "sqp_iters_mean": float(stats[:, 0].mean()), "admm_iters_mean": float(stats[:, 1].mean()),
                    "factorizations_mean": float(stats[:, 5].mean())},
    })
    rec["_kkt"] = kkt
    if backends and bwd:
        rec["backward_backends"] = backward_backends(s, pb, sol, dLdz, flush, max(3, steps // 4))
    if plain and solver in (0, 2) and set(int(m) for m in np.unique(pb.model)) <= set(FAST_MODELS):
        rec["plain_form"] = plain_form(pb, args, flush, ms_f, kkt)
    if e2e:
        hp = {k: (v.cpu().pin_memory() if v is not None else None) for k, v in tensors_from_batch(pb, "cpu").items()}
        ho = {k: v.cpu().pin_memory() for k, v in s.alloc_solution("cpu").items()}
        h2d = sum(v.numel() * v.element_size() for v in hp.values() if v is not None)
        d2h = sum(v.numel() * v.element_size() for v in ho.values())
        for _ in range(max(1, warmup)):
            s.tmpc_solve_host(hp, hp["x0"], ho, z_init_host=hp["z_init"])
        e2e_t = []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t = time.perf_counter()
            s.tmpc_solve_host(hp, hp["x0"], ho, z_init_host=hp["z_init"])
            e2e_t.append(time.perf_counter() - t)
        rec["e2e"] = {"ms": 1e3 * float(np.mean(e2e_t)), "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    s.close()
    return rec


def plain_form(pb, args, flush, persistent_ms, kkt):
    """The plain per-phase form of the same solve (one launch per phase, eager
    and captured as a CUDA graph): the baseline the persistent kernel beats."""
    import torch
    from paper_2606_24039_gb300 import Solver
    sp = Solver.from_batch(pb, device="cuda", solver=7, threads=args.threads)
    solp = sp.alloc_solution("cuda")
    warm = sp.z_init is not None
    side = torch.cuda.Stream()
    stream = torch.cuda.current_stream()

    def pstep():
        if warm:
            solp["z"].copy_(sp.z_init)
            for k in ("xi", "y_eq", "y_ineq"):
                solp[k].zero_()
        sp.tmpc_solve(sp.x0, solp, warm_start=warm)

    for _ in range(2):
        pstep()
    torch.cuda.synchronize()

    def time_fn(fn, n=3):
        ts = []
        for _ in range(n):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
    out = {"eager_ms": eager_ms, "graph_ms": graph_ms, "persistent_ms": persistent_ms,
           "launches_per_step": groups_p * (2 + pb.opts.max_sqp * (2 + pb.opts.max_admm)),
           "kkt_median": float(np.median(kp)), "kkt_median_persistent": float(np.median(kkt)),
           "speedup_vs_eager": eager_ms / persistent_ms, "speedup_vs_graph": graph_ms / persistent_ms}
    del g
    sp.close()
    return out


def closed_loop(pb, H, flush, steps=3):
    """Closed-loop MPC episodes of the linear-system RL problem: H steps, each an
    MPC solve of the whole batch through the differentiable layer, the first
    control applied to x+ = A x + B u + b; the reward -(sum ||x||^2 + ||u||^2) is
    differentiated with respect to theta = diag(Q) by autograd (the backward
    chains every step's implicit-differentiation pass)."""
    import torch
    from paper_2606_24039_gb300 import Solver, solve_ocp
    s = Solver.from_batch(pb, device="cuda")
    A = torch.tensor(pb.extra["A"], dtype=torch.float32, device="cuda")
    Bm = torch.tensor(pb.extra["B"], dtype=torch.float32, device="cuda")
    b = torch.tensor(pb.extra["b"], dtype=torch.float32, device="cuda")
    Rd = torch.tensor(pb.Rd, dtype=torch.float32, device="cuda")
    ref = torch.zeros((pb.B, pb.N_max + 1, pb.n), device="cuda")
    lo = torch.tensor(pb.lo, dtype=torch.float32, device="cuda")
    hi = torch.tensor(pb.hi, dtype=torch.float32, device="cuda")
    x0 = torch.tensor(pb.x0, dtype=torch.float32, device="cuda")
    nx = pb.nx

    def episode(grad):
        theta = torch.tensor(pb.extra["theta"], dtype=torch.float32, device="cuda", requires_grad=grad)
        x, R = x0, torch.zeros((), device="cuda")
        for _ in range(H):
            Qd = (2.0 * theta)[None, None, :].expand(pb.B, pb.N_max + 1, nx).contiguous()
            z, _, _ = solve_ocp(s, x, Qd, Rd, ref, lo, hi)
            u = z[:, 0, nx:]
            R = R - (x * x).sum() - (u * u).sum()
            x = x @ A.T + u @ Bm.T + b
        if grad:
            R.backward()
        return R

    for _ in range(2):
        episode(True)
    torch.cuda.synchronize()
    out = {}
    for key, grad in (("fwd", False), ("fwd_bwd", True)):
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t = time.perf_counter()
            with torch.set_grad_enabled(grad):
                episode(grad)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t)
        ms = 1e3 * float(np.mean(ts))
        out[key] = {"ms_per_episode": ms, "solves_per_s": pb.B * H / (ms * 1e-3)}
    s.close()
    return {"H": H, "batch": pb.B, **out,
            "note": "wall clock per episode (host loop over H MPC solves, each through TmpcFunction)"}


def converged_batch(name, pb):
    """The workload solved to the tolerance 1e-5 (early exit at eps_abs = eps_rel =
    eps_c = 1e-5, <= 1000 ADMM iterations per QP, <= 10 SQP iterations for the
    linear problems and <= 20 otherwise)."""
    import dataclasses
    pb.opts = dataclasses.replace(pb.opts, early_exit=1, eps_abs=1e-5, eps_rel=1e-5, eps_c=1e-5, max_admm=1000,
                                  max_sqp=10 if name in LINEAR else 20, check_every=25)
    return pb


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
    from paper_2606_24039_gb300 import build
    build.build()
    peak = fp32_peak(local)
    fma_measured = fp32_probe()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    pb = workload(args, rank, world=world)
    suite = not args.no_suite and args.workload == "uneven" and world == 1
    if world > 1:
        dist.barrier()
    with Clocks(local, args.clocks_csv) as clk:
        t0 = time.time()
        head = measure(args.workload, pb, args, peak, flush, args.steps, args.warmup,
                       autotune=(args.solver == 0 and not args.no_autotune), plain=not args.no_plain,
                       e2e=not args.skip_e2e, bwd=not args.skip_bwd, solver=args.solver, world=world,
                       backends=suite)
        t1 = time.time()
        subs, conv = {}, {}
        if suite:
            for name in SUITE:
                spb = workload(args, rank, name, world=world)
                r = measure(name, spb, args, peak, flush, max(3, args.steps // 4), max(3, args.warmup // 2),
                            autotune=(name == "racing"), bwd=True)
                if name == "linear_rl":
                    r["closed_loop"] = closed_loop(spb, 50, flush)
                r.pop("_kkt", None)
                subs[name] = r
            for name in ("uneven",) + SUITE:
                cpb = converged_batch(name, workload(args, rank, name, world=world))
                r = measure(name, cpb, args, peak, flush, 2, 1, bwd=False)
                kkt = r.pop("_kkt")
                conv[name] = {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                              "frac_kkt_le_1e-5": float(np.mean(kkt <= 1e-5)),
                              "solves_at_1e-5_per_s": float(np.sum(kkt <= 1e-5)) / (r["ms_per_step"] * 1e-3),
                              "kkt_median": float(np.median(kkt)), "kkt_p90": float(np.percentile(kkt, 90)),
                              "sqp_iters_mean": r["quality"]["sqp_iters_mean"],
                              "admm_iters_mean": r["quality"]["admm_iters_mean"],
                              "status_counts": r["quality"]["status_counts"], "config": r["config"]["workload"]}
        t2 = time.time()
    head.pop("_kkt", None)
    clocks = clk.summary(t0, t1)
    clocks_all = clk.summary(t0, t2)
    ms_f = head["ms_per_step"]
    ms_fb = head["fwd_bwd"]["ms_per_step"] if head["fwd_bwd"] else float("nan")
    ms_e2e = head["e2e"]["ms"] if "e2e" in head else float("nan")
    if world > 1:   # the slowest rank sets the job time (no collective on the data path)
        from paper_2606_24039_gb300.shard import max_over_ranks
        ms_f, ms_fb, ms_e2e = (max_over_ranks(v, device="cuda") for v in (ms_f, ms_fb, ms_e2e))
    total = pb.B * world
    if rank == 0:
        line = {
            "metric": METRIC, "value": total / (ms_f * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_f, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_of(args, pb),
            "fwd_bwd": {"value": total / (ms_fb * 1e-3), "unit": UNIT, "ms_per_step": ms_fb},
            "clocks": clocks,
            "e2e": ({"value": total / (ms_e2e * 1e-3), "unit": UNIT,
                     "h2d_bytes_per_step": head["e2e"]["h2d_bytes_per_step"],
                     "d2h_bytes_per_step": head["e2e"]["d2h_bytes_per_step"]} if "e2e" in head else None),
            "gpu_launches": head["gpu_launches"],
            "roofline": head["roofline"],
            "group_times": head["group_times"],
            "cpu_baseline": cpu_base,
            "plain_form": head.get("plain_form"),
            "autotune": head.get("autotune"),
            "quality": head["quality"],
            "backward_backends": head.get("backward_backends"),
            "fp32_peak": {"tflops": peak[0], "sms": peak[1], "sm_max_mhz": peak[2],
                          "measured_tflops": fma_measured,
                          "measured_note": "FMA-chain probe (tmpc_fp32_fma_probe), at the clock of the moment"},
        }
        if suite:
            line["workloads"] = subs
            line["at_1e-5"] = conv
            line["clocks_suite"] = clocks_all
        print(json.dumps(line), flush=True)
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
