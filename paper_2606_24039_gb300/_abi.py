"""ctypes mirror of include/tmpc.h.  Argument marshalling only: every step of
the solver runs in the CUDA library; nothing here computes."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_float_p = ctypes.POINTER(ctypes.c_float)
c_int_p = ctypes.POINTER(ctypes.c_int32)

TMPC_STATS = 10
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory",
          4: "not set up", 5: "unsupported"}
INST_STATUS = {0: "ok", 1: "max_iter", 2: "not_pd", 3: "nan", 4: "invalid"}
STATIC_SCRATCH_BYTES = 64 << 20


class Dims(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("N_max", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("nu", ctypes.c_int32), ("ng", ctypes.c_int32), ("n_dyn", ctypes.c_int32),
                ("n_track", ctypes.c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_float), ("rho0", ctypes.c_float), ("rho_min", ctypes.c_float),
                ("rho_max", ctypes.c_float), ("alpha", ctypes.c_float),
                ("eps_abs", ctypes.c_float), ("eps_rel", ctypes.c_float), ("eps_c", ctypes.c_float),
                ("eps_g", ctypes.c_float), ("ls_eta", ctypes.c_float),
                ("k_rho_iter", ctypes.c_int32), ("k_rho_ratio", ctypes.c_float),
                ("max_sqp", ctypes.c_int32), ("max_admm", ctypes.c_int32), ("n_ls", ctypes.c_int32),
                ("newton_steps", ctypes.c_int32), ("early_exit", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("bwd_rho", ctypes.c_float),
                ("bwd_sigma", ctypes.c_float), ("bwd_iters", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("force_pivot_failure", ctypes.c_int32), ("wait_polls", ctypes.c_int32),
                ("force_wait_timeout", ctypes.c_int32), ("bwd_solver", ctypes.c_int32),
                ("exact_hessian", ctypes.c_int32), ("bwd_gamma", ctypes.c_float)]


class Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_void_p), ("model", ctypes.c_void_p), ("Qd", ctypes.c_void_p),
                ("Rd", ctypes.c_void_p), ("Wd", ctypes.c_void_p), ("ref", ctypes.c_void_p),
                ("lin", ctypes.c_void_p), ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p),
                ("gamma2", ctypes.c_void_p), ("gamma1", ctypes.c_void_p), ("dyn", ctypes.c_void_p),
                ("track", ctypes.c_void_p), ("scale", ctypes.c_void_p)]


class Solution(ctypes.Structure):
    _fields_ = [("z", ctypes.c_void_p), ("xi", ctypes.c_void_p), ("y_eq", ctypes.c_void_p),
                ("y_ineq", ctypes.c_void_p), ("status", ctypes.c_void_p), ("stats", ctypes.c_void_p)]


class Grads(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_void_p), ("Qd", ctypes.c_void_p), ("Rd", ctypes.c_void_p),
                ("Wd", ctypes.c_void_p), ("ref", ctypes.c_void_p), ("lin", ctypes.c_void_p),
                ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p), ("gamma2", ctypes.c_void_p),
                ("gamma1", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("count", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("cluster", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("ms", ctypes.c_float), ("ms_default", ctypes.c_float)]


EXPORTS = ["tmpc_default_options", "tmpc_setup", "tmpc_update_params", "tmpc_set_options",
           "tmpc_solve", "tmpc_backward", "tmpc_solve_host", "tmpc_destroy",
           "tmpc_status_string", "tmpc_last_error", "tmpc_solve_static", "tmpc_autotune"]

_lib = None


class GroupTime(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("form", ctypes.c_int32), ("count", ctypes.c_int32),
                ("fwd_ms", ctypes.c_float), ("bwd_ms", ctypes.c_float)]


class TmpcError(RuntimeError):
    pass


def load(path: str | None = None):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.lib_path()
    if not os.path.exists(path):
        raise TmpcError(f"CUDA solver library not built: {path} is missing "
                        "(run paper_2606_24039_gb300.build.build())")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.tmpc_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.tmpc_default_options.restype = None
    lib.tmpc_setup.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Dims), ctypes.POINTER(Options),
                               ctypes.POINTER(Params)]
    lib.tmpc_setup.restype = ctypes.c_int
    lib.tmpc_update_params.argtypes = [vp, ctypes.POINTER(Params)]
    lib.tmpc_update_params.restype = ctypes.c_int
    lib.tmpc_set_options.argtypes = [vp, ctypes.POINTER(Options)]
    lib.tmpc_set_options.restype = ctypes.c_int
    lib.tmpc_solve.argtypes = [vp, vp, ctypes.POINTER(Solution), ctypes.c_int32, vp]
    lib.tmpc_solve.restype = ctypes.c_int
    lib.tmpc_backward.argtypes = [vp, vp, ctypes.POINTER(Solution), vp, vp, ctypes.POINTER(Grads), vp]
    lib.tmpc_backward.restype = ctypes.c_int
    lib.tmpc_solve_host.argtypes = [vp, ctypes.POINTER(Params), vp, vp, ctypes.POINTER(Solution), vp]
    lib.tmpc_solve_host.restype = ctypes.c_int
    lib.tmpc_solve_static.argtypes = [ctypes.POINTER(Dims), ctypes.POINTER(Options), ctypes.POINTER(Params), vp,
                                      ctypes.POINTER(Solution), ctypes.c_int32, vp]
    lib.tmpc_solve_static.restype = ctypes.c_int
    lib.tmpc_autotune.argtypes = [vp, vp, ctypes.POINTER(Solution), ctypes.c_int32, ctypes.c_int32,
                                  ctypes.POINTER(TuneResult), vp]
    lib.tmpc_autotune.restype = ctypes.c_int
    lib.tmpc_group_times.argtypes = [vp, ctypes.POINTER(GroupTime), ctypes.POINTER(ctypes.c_int32)]
    lib.tmpc_group_times.restype = ctypes.c_int
    lib.tmpc_fp32_fma_probe.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    lib.tmpc_fp32_fma_probe.restype = ctypes.c_int
    lib.tmpc_destroy.argtypes = [vp]
    lib.tmpc_destroy.restype = None
    lib.tmpc_status_string.argtypes = [ctypes.c_int]
    lib.tmpc_status_string.restype = ctypes.c_char_p
    lib.tmpc_last_error.argtypes = []
    lib.tmpc_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def ls_history(stats_row, n_sqp):
    """Line-search steps of the first min(n_sqp, 12) SQP iterations decoded from
    stats[8:10] (2^-k per 4-bit code k, 0.0 for code 15)."""
    out = []
    for j in range(min(int(n_sqp), 12)):
        code = (int(stats_row[8 + j // 6]) >> (4 * (j % 6))) & 15
        out.append(0.0 if code == 15 else 2.0 ** (-code))
    return out


def check(code: int, what: str):
    if code != 0:
        lib = load()
        msg = lib.tmpc_status_string(code).decode()
        extra = lib.tmpc_last_error().decode()
        raise TmpcError(f"{what} failed: {msg}" + (f" ({extra})" if extra and code in (1, 2) else ""))


def default_options() -> Options:
    o = Options()
    load().tmpc_default_options(ctypes.byref(o))
    return o
