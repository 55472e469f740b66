"""Torch-facing binding of the C ABI (include/tmpc.h).

PyTorch supplies device memory and streams only; every step of the solver
(linearisation, factorisation, ADMM, line search, backward) runs in the CUDA
library.  The same function names as the ABI are exposed on `Solver`.
"""
from __future__ import annotations

import ctypes

import torch

from . import _abi

PARAM_KEYS = ("Qd", "Rd", "Wd", "ref", "lin", "lo", "hi", "gamma2", "gamma1", "dyn", "track", "scale")
GRAD_KEYS = ("x0", "Qd", "Rd", "Wd", "ref", "lin", "lo", "hi", "gamma2", "gamma1")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def options_from(opts=None, **overrides) -> _abi.Options:
    """ABI options from defaults, an object with matching attribute names, and overrides."""
    o = _abi.default_options()
    names = [f[0] for f in _abi.Options._fields_]
    if opts is not None:
        for k in names:
            if hasattr(opts, k):
                setattr(o, k, getattr(opts, k))
    for k, v in overrides.items():
        if k not in names:
            raise KeyError(k)
        setattr(o, k, v)
    return o


def tensors_from_batch(pb, device="cuda") -> dict:
    """Device tensors (FP32 / int32, contiguous) of a problem batch object with
    the attributes of the ABI parameter struct (N, model, x0, Qd, ...)."""
    f = lambda a: None if a is None else torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
    out = {k: f(getattr(pb, k, None)) for k in PARAM_KEYS}
    out["x0"] = f(pb.x0)
    out["z_init"] = f(getattr(pb, "z_init", None))
    out["N"] = torch.as_tensor(pb.N, dtype=torch.int32).contiguous().to(device)
    out["model"] = torch.as_tensor(pb.model, dtype=torch.int32).contiguous().to(device)
    return out


class Solver:
    """One C-ABI handle: workspace for a fixed layout (B, N_max, nx, nu, ng)."""

    def __init__(self, dims: dict, params: dict, options: _abi.Options | None = None):
        self.lib = _abi.load()
        self.dims = _abi.Dims(dims["batch"], dims["N_max"], dims["nx"], dims["nu"], dims["ng"],
                              dims["n_dyn"], dims.get("n_track", 0))
        self.options = options if options is not None else _abi.default_options()
        self._params = {}
        self._pstruct = self._make_params(params)
        self.handle = ctypes.c_void_p()
        _abi.check(self.lib.tmpc_setup(ctypes.byref(self.handle), ctypes.byref(self.dims),
                                       ctypes.byref(self.options), ctypes.byref(self._pstruct)),
                   "tmpc_setup")

    @classmethod
    def from_batch(cls, pb, device="cuda", **overrides):
        t = tensors_from_batch(pb, device)
        dims = dict(batch=pb.B, N_max=pb.N_max, nx=pb.nx, nu=pb.nu, ng=pb.ng, n_dyn=pb.n_dyn,
                    n_track=pb.n_track)
        s = cls(dims, t, options_from(pb.opts, **overrides))
        s.x0 = t["x0"]
        s.z_init = t["z_init"]
        return s

    def _make_params(self, params):
        keep = {}
        for k in ("N", "model") + PARAM_KEYS:
            v = params.get(k)
            if v is not None:
                if not v.is_contiguous():
                    raise ValueError(f"parameter {k} must be contiguous")
                keep[k] = v
        self._params = keep
        p = _abi.Params()
        for k in ("N", "model") + PARAM_KEYS:
            v = keep.get(k)
            setattr(p, k, None if v is None else v.data_ptr())
        return p

    @property
    def B(self):
        return self.dims.batch

    def _shapes(self):
        d = self.dims
        T = d.N_max + 1
        n = d.nx + d.nu
        return dict(z=(d.batch, T, n), xi=(d.batch, T, d.ng), y_eq=(d.batch, T, d.nx),
                    y_ineq=(d.batch, T, d.ng))

    def alloc_solution(self, device="cuda"):
        sh = self._shapes()
        out = {k: torch.zeros(v, dtype=torch.float32, device=device) for k, v in sh.items()}
        out["status"] = torch.zeros(self.B, dtype=torch.int32, device=device)
        out["stats"] = torch.zeros((self.B, _abi.TMPC_STATS), dtype=torch.float32, device=device)
        return out

    @staticmethod
    def _sol_struct(sol):
        return _abi.Solution(*[sol[k].data_ptr() if sol.get(k) is not None else None
                               for k in ("z", "xi", "y_eq", "y_ineq", "status", "stats")])

    def tmpc_update_params(self, params: dict):
        merged = dict(self._params)
        merged.update({k: v for k, v in params.items() if k in PARAM_KEYS})
        self._pstruct = self._make_params(merged)
        _abi.check(self.lib.tmpc_update_params(self.handle, ctypes.byref(self._pstruct)), "tmpc_update_params")

    def tmpc_set_options(self, options: _abi.Options):
        _abi.check(self.lib.tmpc_set_options(self.handle, ctypes.byref(options)), "tmpc_set_options")
        self.options = options

    def tmpc_solve(self, x0, sol=None, warm_start=False, stream=None, z_init=None):
        """Forward solve.  warm_start reads sol as the initial primal-dual guess;
        z_init (device tensor shaped like sol["z"]) is copied into sol["z"] as the
        initial primal guess with zero slacks and multipliers."""
        if sol is None:
            sol = self.alloc_solution(x0.device)
        if z_init is not None:
            sol["z"].copy_(z_init)
            sol["xi"].zero_()
            sol["y_eq"].zero_()
            sol["y_ineq"].zero_()
            warm_start = True
        s = self._sol_struct(sol)
        _abi.check(self.lib.tmpc_solve(self.handle, ctypes.c_void_p(x0.data_ptr()), ctypes.byref(s),
                                       1 if warm_start else 0, _stream_ptr(stream)), "tmpc_solve")
        return sol

    def tmpc_backward(self, x0, sol, dL_dz, dL_dxi=None, grads=None, stream=None):
        if grads is None:
            grads = {k: torch.zeros_like(self._params[k] if k != "x0" else x0)
                     for k in GRAD_KEYS if (k == "x0" or self._params.get(k) is not None)}
        g = _abi.Grads(*[grads[k].data_ptr() if grads.get(k) is not None else None for k in GRAD_KEYS])
        s = self._sol_struct(sol)
        _abi.check(self.lib.tmpc_backward(self.handle, ctypes.c_void_p(x0.data_ptr()), ctypes.byref(s),
                                          ctypes.c_void_p(dL_dz.contiguous().data_ptr()),
                                          None if dL_dxi is None else ctypes.c_void_p(dL_dxi.contiguous().data_ptr()),
                                          ctypes.byref(g), _stream_ptr(stream)), "tmpc_backward")
        return grads

    def tmpc_autotune(self, x0, init=None, reps=3, trial_sqp=0, stream=None):
        """Time each launch form of every model group on x0 and keep the fastest
        (synchronous).  init: a solution dict read as the trials' warm start (not
        written); None starts cold.  Returns one dict per group (fields of
        tmpc_tune_result)."""
        res = (_abi.TuneResult * 4)()
        si = None if init is None else self._sol_struct(init)
        _abi.check(self.lib.tmpc_autotune(self.handle, ctypes.c_void_p(x0.data_ptr()),
                                          None if si is None else ctypes.byref(si), int(reps),
                                          int(trial_sqp), res, _stream_ptr(stream)), "tmpc_autotune")
        # entries of absent groups are left as zeroed by ctypes (count 0)
        return [{f: getattr(r, f) for f, _ in _abi.TuneResult._fields_} for r in res if r.count > 0]

    def tmpc_group_times(self):
        """Device milliseconds of the last forward / backward launch of each model
        group (CUDA events on the launching streams); list of dicts."""
        res = (_abi.GroupTime * 5)()
        n = ctypes.c_int32(0)
        _abi.check(self.lib.tmpc_group_times(self.handle, res, ctypes.byref(n)), "tmpc_group_times")
        return [{f: getattr(r, f) for f, _ in _abi.GroupTime._fields_} for r in res[:n.value]]

    def tmpc_solve_host(self, host_params: dict, x0_host, out_host: dict, stream=None, z_init_host=None):
        """End-to-end solve from pinned host tensors (copies inside the call)."""
        p = _abi.Params()
        for k in ("N", "model") + PARAM_KEYS:
            v = host_params.get(k)
            setattr(p, k, None if v is None else v.data_ptr())
        s = self._sol_struct(out_host)
        zi = None if z_init_host is None else ctypes.c_void_p(z_init_host.data_ptr())
        _abi.check(self.lib.tmpc_solve_host(self.handle, ctypes.byref(p), ctypes.c_void_p(x0_host.data_ptr()),
                                            zi, ctypes.byref(s), _stream_ptr(stream)), "tmpc_solve_host")
        return out_host

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.tmpc_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tmpc_solve_static(dims: dict, params: dict, x0, sol: dict, options: _abi.Options | None = None,
                      warm_start=False, stream=None):
    """Forward solve through the no-allocation entry point (no handle; scratch in
    the library's static device array).  `sol` must be preallocated (status
    included); raises TmpcError when the batch does not fit the scratch."""
    lib = _abi.load()
    d = _abi.Dims(dims["batch"], dims["N_max"], dims["nx"], dims["nu"], dims["ng"], dims["n_dyn"],
                  dims.get("n_track", 0))
    o = options if options is not None else _abi.default_options()
    p = _abi.Params()
    for k in ("N", "model") + PARAM_KEYS:
        v = params.get(k)
        setattr(p, k, None if v is None else v.data_ptr())
    s = Solver._sol_struct(sol)
    code = lib.tmpc_solve_static(ctypes.byref(d), ctypes.byref(o), ctypes.byref(p), ctypes.c_void_p(x0.data_ptr()),
                                 ctypes.byref(s), 1 if warm_start else 0, _stream_ptr(stream))
    if code != 0:
        raise _abi.TmpcError(f"tmpc_solve_static failed: {lib.tmpc_status_string(code).decode()}"
                             f" ({lib.tmpc_last_error().decode()})")
    return sol


class TmpcFunction(torch.autograd.Function):
    """(z, xi, status) = OCP solve of Algorithm 1 as a function of x0 and the cost
    and bound parameters, with the implicit-differentiation backward of the
    library (Algorithm 2).  Differentiable inputs: x0, Qd, Rd, ref, lo, hi and,
    when given (not None), Wd, lin, gamma2, gamma1; the solver handle carries
    the remaining parameters (dynamics, track).  The forward keeps only the
    solution and the inputs: the backward refactors the adjoint system from
    the solution instead of storing any ADMM iterate."""

    @staticmethod
    def forward(ctx, solver: Solver, x0, Qd, Rd, ref, lo, hi, Wd=None, lin=None, gamma2=None, gamma1=None):
        names = ("Qd", "Rd", "ref", "lo", "hi", "Wd", "lin", "gamma2", "gamma1")
        vals = [None if t is None else t.detach().float().contiguous() for t in (Qd, Rd, ref, lo, hi, Wd, lin, gamma2, gamma1)]
        x0 = x0.detach().float().contiguous()
        params = {k: v for k, v in zip(names, vals) if v is not None}
        solver.tmpc_update_params(params)
        sol = solver.tmpc_solve(x0)
        ctx.solver = solver
        ctx.sol = sol
        ctx.names = [k for k, v in zip(names, vals) if v is not None]
        ctx.given = [v is not None for v in vals]
        ctx.save_for_backward(x0, *[v for v in vals if v is not None])
        ctx.mark_non_differentiable(sol["status"])
        return sol["z"], sol["xi"], sol["status"]

    @staticmethod
    def backward(ctx, dz, dxi, _dstatus):
        x0, *vals = ctx.saved_tensors
        solver = ctx.solver
        solver.tmpc_update_params(dict(zip(ctx.names, vals)))
        g = solver.tmpc_backward(x0, ctx.sol, dz.contiguous().float(),
                                 None if dxi is None else dxi.contiguous().float())
        out = [g["x0"]]
        for k, given in zip(("Qd", "Rd", "ref", "lo", "hi", "Wd", "lin", "gamma2", "gamma1"), ctx.given):
            out.append(g.get(k) if given else None)
        return (None, *out)


def solve_ocp(solver: Solver, x0, Qd, Rd, ref, lo, hi, Wd=None, lin=None, gamma2=None, gamma1=None):
    """Differentiable forward solve; returns (z, xi, status)."""
    return TmpcFunction.apply(solver, x0, Qd, Rd, ref, lo, hi, Wd, lin, gamma2, gamma1)
