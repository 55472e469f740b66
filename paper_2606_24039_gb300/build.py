"""Build the CUDA library (C ABI of include/tmpc.h) in-tree with nvcc for
sm_103a.  The shared object lands in paper_2606_24039_gb300/lib/ and is
git-ignored; it must be rebuilt on every machine (x86 here, aarch64 on the
GPU hosts)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
LIBNAME = "libtmpc.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# the heavy kernels sit in translation units of their own so that they compile in parallel
SOURCES = ["tmpc_api.cu", "tmpc_probe.cu", "tmpc_generic_fwd.cu", "tmpc_generic_bwd.cu", "tmpc_fast.cu",
           "tmpc_fast_di.cu", "tmpc_fast_bicycle.cu", "tmpc_fast_quad.cu"]


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the solver library")


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "tmpc.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source into one shared library; returns its path."""
    os.makedirs(LIBDIR, exist_ok=True)
    out = lib_path()
    if not force and not _stale(out):
        return out
    nvcc = nvcc_path()
    objs = []
    procs = []
    for src in SOURCES:
        obj = os.path.join(LIBDIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, "-O3", "-lineinfo", "-std=c++17", *ARCH, "-Xcompiler", "-fPIC",
               "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.append("-Xptxas=-v")
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    for src, p in procs:
        log, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{log}")
        if verbose and log:
            print(log, file=sys.stderr)
    tmp = out + ".tmp"
    cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
