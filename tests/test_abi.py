"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function declared in include/tmpc.h, and rejects bad arguments before
touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_24039_gb300 import build, load
    build.build()
    return load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tmpc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tmpc_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["tmpc_setup", "tmpc_solve", "tmpc_backward", "tmpc_destroy", "tmpc_solve_host",
              "tmpc_update_params", "tmpc_status_string"]:
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_setup_rejects_bad_arguments_without_a_gpu(lib):
    from paper_2606_24039_gb300 import _abi
    h = ctypes.c_void_p()
    d = _abi.Dims(4, 10, 4, 2, 4, 1, 0)
    o = _abi.default_options()
    p = _abi.Params()
    # null parameter pointers
    assert lib.tmpc_setup(ctypes.byref(h), ctypes.byref(d), ctypes.byref(o), ctypes.byref(p)) == 1
    assert h.value is None
    # null handle pointer / dims
    assert lib.tmpc_setup(None, ctypes.byref(d), ctypes.byref(o), ctypes.byref(p)) == 1
    assert lib.tmpc_setup(ctypes.byref(h), None, ctypes.byref(o), ctypes.byref(p)) == 1
    # dimensions beyond the compiled limits
    d2 = _abi.Dims(4, 10, 70, 10, 4, 1, 0)
    assert lib.tmpc_setup(ctypes.byref(h), ctypes.byref(d2), ctypes.byref(o), ctypes.byref(p)) == 5
    # empty batch, empty horizon
    for bad in (_abi.Dims(0, 10, 4, 2, 4, 1, 0), _abi.Dims(4, 0, 4, 2, 4, 1, 0)):
        assert lib.tmpc_setup(ctypes.byref(h), ctypes.byref(bad), ctypes.byref(o), ctypes.byref(p)) == 1
    # bad options
    o2 = _abi.default_options()
    o2.alpha = 2.5
    assert lib.tmpc_setup(ctypes.byref(h), ctypes.byref(d), ctypes.byref(o2), ctypes.byref(p)) == 1
    for field, value in (("solver", 8), ("threads", 48), ("threads", 512), ("n_ls", 17), ("max_admm", 0),
                         ("bwd_solver", 4), ("bwd_solver", -1)):
        o3 = _abi.default_options()
        setattr(o3, field, value)
        assert lib.tmpc_setup(ctypes.byref(h), ctypes.byref(d), ctypes.byref(o3), ctypes.byref(p)) == 1, field
    assert abs(_abi.default_options().bwd_gamma - 1e4) < 1e-3


def test_backward_options_are_validated_before_any_device_work(lib):
    """The option check alone rejects a backward solver outside 0..3 and a reduced
    adjoint QP (3) with a non-positive or infinite penalty or with the exact
    Hessian: the no-allocation entry point, given well-formed parameters and a
    batch too large for its scratch, stops at the option check for these (no
    scratch message) and reaches the capacity check with the defaults."""
    from paper_2606_24039_gb300 import _abi
    d = _abi.Dims(4096, 30, 6, 2, 5, 4, 800)
    fake = 0x10000
    p = _abi.Params(*([fake] * 13))
    s = _abi.Solution(*([fake] * 6))

    def call(o):
        code = lib.tmpc_solve_static(ctypes.byref(d), ctypes.byref(o), ctypes.byref(p), fake, ctypes.byref(s), 0, None)
        return code, lib.tmpc_last_error().decode()

    code, msg = call(_abi.default_options())
    assert code == 1 and "static scratch" in msg
    for bwd, exact, gamma in ((4, 0, 1e4), (-1, 0, 1e4), (3, 1, 1e4), (3, 0, 0.0), (3, 0, float("inf"))):
        o = _abi.default_options()
        o.bwd_solver, o.exact_hessian, o.bwd_gamma = bwd, exact, gamma
        code, msg = call(o)
        assert code == 1 and "static scratch" not in msg, (bwd, exact, gamma)
    o = _abi.default_options()
    o.bwd_solver = 3
    assert "static scratch" in call(o)[1]
    # calls on a null handle
    assert lib.tmpc_solve(None, None, None, 0, None) == 4
    assert lib.tmpc_backward(None, None, None, None, None, None, None) == 4
    assert lib.tmpc_autotune(None, None, None, 1, 1, None, None) == 4
    assert ctypes.sizeof(_abi.TuneResult) == 32
    lib.tmpc_destroy(None)
    assert lib.tmpc_status_string(0) == b"ok"


def test_default_options_follow_the_paper(lib):
    from paper_2606_24039_gb300 import _abi
    o = _abi.default_options()
    assert abs(o.sigma - 1e-6) < 1e-12 and abs(o.rho0 - 0.1) < 1e-7
    assert o.k_rho_iter == 25 and abs(o.k_rho_ratio - 5.0) < 1e-7
    assert abs(o.rho_min - 1e-6) < 1e-12 and abs(o.rho_max - 1e6) < 1
    assert abs(o.ls_eta - 0.4) < 1e-7


def test_static_entry_validates_before_touching_the_device(lib):
    """tmpc_solve_static rejects null arguments and a batch whose scratch exceeds
    the static array before any CUDA call (the pointers below are never read)."""
    from paper_2606_24039_gb300 import _abi
    d = _abi.Dims(4096, 30, 6, 2, 5, 4, 800)
    o = _abi.default_options()
    fake = 0x10000
    p = _abi.Params(*([fake] * 13))
    s = _abi.Solution(*([fake] * 6))
    assert lib.tmpc_solve_static(None, ctypes.byref(o), ctypes.byref(p), fake, ctypes.byref(s), 0, None) == 1
    assert lib.tmpc_solve_static(ctypes.byref(d), ctypes.byref(o), ctypes.byref(p), None, ctypes.byref(s), 0, None) == 1
    o3 = _abi.default_options()
    o3.solver = 2
    assert lib.tmpc_solve_static(ctypes.byref(d), ctypes.byref(o3), ctypes.byref(p), fake, ctypes.byref(s), 0, None) == 1
    assert lib.tmpc_solve_static(ctypes.byref(d), ctypes.byref(o), ctypes.byref(p), fake, ctypes.byref(s), 0, None) == 1
    msg = lib.tmpc_last_error().decode()
    assert "static scratch holds %d bytes" % _abi.STATIC_SCRATCH_BYTES in msg


def test_tune_result_mirror_matches_the_header():
    """The ctypes mirror of tmpc_tune_result has the header's fields, in order and type."""
    from paper_2606_24039_gb300 import _abi
    src = open(os.path.join(ROOT, "include", "tmpc.h")).read()
    end = src.index("} tmpc_tune_result;")
    body = src[src.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(int32_t|float)\s+(\w+);", body)
    ctype = {"int32_t": ctypes.c_int32, "float": ctypes.c_float}
    assert [(n, ctype[t]) for t, n in fields] == list(_abi.TuneResult._fields_)


def test_static_entry_rejects_a_workspace_beyond_int_offsets(lib):
    """A horizon whose per-instance workspace exceeds 2^31 floats is rejected
    before any CUDA call (the layout is computed in 64-bit; it used to wrap)."""
    from paper_2606_24039_gb300 import _abi
    d = _abi.Dims(1, 10873336, 6, 2, 5, 4, 800)
    o = _abi.default_options()
    fake = 0x10000
    p = _abi.Params(*([fake] * 13))
    s = _abi.Solution(*([fake] * 6))
    assert lib.tmpc_solve_static(ctypes.byref(d), ctypes.byref(o), ctypes.byref(p), fake, ctypes.byref(s), 0, None) == 1
    assert "exceeds 2^31 floats" in lib.tmpc_last_error().decode()


def test_options_mirror_matches_the_header():
    """The ctypes mirror of tmpc_options has the header's fields, in order and type."""
    from paper_2606_24039_gb300 import _abi
    src = open(os.path.join(ROOT, "include", "tmpc.h")).read()
    end = src.index("} tmpc_options;")
    body = src[src.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in re.findall(r"\b(int32_t|float)\s+([^;]+);", body):
        for name in decl[1].split(","):
            fields.append((name.strip(), {"int32_t": ctypes.c_int32, "float": ctypes.c_float}[decl[0]]))
    assert fields == list(_abi.Options._fields_)


def test_group_time_mirror_matches_the_header():
    from paper_2606_24039_gb300 import _abi
    src = open(os.path.join(ROOT, "include", "tmpc.h")).read()
    end = src.index("} tmpc_group_time;")
    body = src[src.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(int32_t|float)\s+(\w+);", body)
    ctype = {"int32_t": ctypes.c_int32, "float": ctypes.c_float}
    assert [(n, ctype[t]) for t, n in fields] == list(_abi.GroupTime._fields_)
    lib = _abi.load()
    assert lib.tmpc_group_times(None, None, None) == 4


def test_params_mirror_matches_the_header():
    """The ctypes mirror of tmpc_params lists the header's pointers, in order."""
    from paper_2606_24039_gb300 import _abi
    src = open(os.path.join(ROOT, "include", "tmpc.h")).read()
    end = src.index("} tmpc_params;")
    body = src[src.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\bconst\s+(?:int32_t|float)\s*\*\s*(\w+);", body)
    assert names == [f for f, _ in _abi.Params._fields_]
    assert names[-1] == "scale"
