"""Host logic of bench.py that needs no GPU: the kernel-launch count it reports
(gpu_launches) and the kernel it names in the roofline, per launch form."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402

bench = pytest.importorskip("bench")


def test_launches_follow_the_launch_form():
    pb = w.racing(B=4, N=50)
    bic = w.MODEL_BICYCLE
    # backward: the CTA pass, the sweep kernel of the direct solve, the finishing pass
    assert bench.launches_per_step(pb, 0) == (1, 3)
    assert bench.launches_per_step(pb, 1) == (1, 1)                    # generic kernel
    assert bench.launches_per_step(pb, 0, {bic: 4}) == (1, 1)          # warp LDL': generic backward
    plain = 2 + pb.opts.max_sqp * (2 + pb.opts.max_admm)
    assert bench.launches_per_step(pb, 0, {bic: 7}) == (plain, 3)      # one launch per phase
    assert bench.launches_per_step(pb, 0, {bic: 6}) == (1, 1)          # cluster: sweeps on its first warp
    assert plain == 522


def test_launches_of_a_mixed_batch():
    pb = w.uneven(B=64, seed=3)
    models = set(int(m) for m in np.unique(pb.model))
    fast = models & set(bench.FAST_MODELS)
    fwd, bwd = bench.launches_per_step(pb, 0)
    assert fwd == len(fast) and bwd == 3 * len(fast)
    # warp LDL' groups share one generic backward launch
    fwd, bwd = bench.launches_per_step(pb, 0, {m: 4 for m in fast})
    assert fwd == len(fast) and bwd == 1


def test_kernel_names_per_form():
    pb = w.racing(B=4, N=50)
    bic = w.MODEL_BICYCLE
    assert bench.kernel_name(pb, 0) == "fast::solve_kernel<MODEL_BICYCLE, kCR>"
    assert bench.kernel_name(pb, 0, {bic: 6}) == "fast::solve_kernel_cluster<MODEL_BICYCLE, kCR>"
    assert bench.kernel_name(pb, 0, {bic: 4}) == "fast::solve_kernel<MODEL_BICYCLE, kLDL>"
    assert bench.kernel_name(pb, 1) == "solve_kernel (generic)"
    assert bench.kernel_name(w.tracking(B=2), 0) == "solve_kernel (generic)"


def test_ranks_take_balanced_shards_of_one_job_batch():
    """Under torchrun every rank draws the same job batch (world x the one-GPU
    batch) and takes its longest-processing-time-first shard: the shards cover
    the job batch exactly once and their (N+1) n^2 work is balanced."""
    import argparse
    from paper_2606_24039_gb300.shard import instance_work
    args = argparse.Namespace(workload="uneven", batch=64, horizon=0)
    parts = [bench.workload(args, r, world=3) for r in range(3)]
    full = bench.make_batch("uneven", 64 * 3, 0, bench.WORKLOADS["uneven"][3])
    key = lambda pb: sorted(map(tuple, np.round(pb.x0, 12)))
    assert sorted(sum((key(p) for p in parts), [])) == key(full)
    n = lambda pb: np.array([sum(w.model_dims(int(m), pb.nx, pb.nu, pb.ng)[:2]) for m in pb.model])
    loads = [float(instance_work(p.N, n(p)).sum()) for p in parts]
    assert max(loads) - min(loads) <= float(instance_work(full.N, n(full)).max())
