"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every entry point declared in include/ccg.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1204_0069_gb300 import build
    return build.build()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+(ccg_[a-z0-9_]+)\s*\(",
                                src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ["ccg_create", "ccg_solve", "ccg_solve_block", "ccg_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_lists_all_exports(libpath):
    from paper_1204_0069_gb300 import ccg
    assert set(ccg.EXPORTED) == set(declared_functions())


def test_status_strings_and_version(libpath):
    from paper_1204_0069_gb300 import ccg
    assert ccg.status_string(0) == "CCG_OK"
    assert ccg.status_string(-5) == "CCG_ERR_TIMEOUT"
    assert ccg.version().startswith("ccg-gb300")


def test_config_defaults(libpath):
    from paper_1204_0069_gb300 import ccg
    cfg = ccg.Config()
    ccg.lib().ccg_config_init(ctypes.byref(cfg))
    assert cfg.rank_tol == 1e-12 and cfg.x0_spread == 1.0 and cfg.residual_replacement == 1
    assert cfg.precision == ccg.FP64 and cfg.mixed_method == ccg.MIXED_AUTO
    assert cfg.cheb_degree == 0 and cfg.cheb_ratio == 0.0 and cfg.batch_autotune == 1


@pytest.mark.parametrize("field,value", [
    ("rank_tol", 0.0), ("rank_tol", -1.0), ("barrier_timeout_ms", 0.0),
    ("precision", 5), ("precision", -1), ("max_ctas", -1), ("inner_tol", -1e-3),
    ("max_outer", -1), ("explicit_residual", 2), ("batch_autotune", 2),
    ("mixed_method", 3), ("cheb_degree", -1), ("cheb_degree", 1025),
    ("cheb_ratio", 1.0), ("cheb_ratio", -0.5)])
def test_create_rejects_each_invalid_field_before_cuda(libpath, field, value):
    """ccg_create validates the whole configuration before its first CUDA
    call, so every out-of-range field gives CCG_ERR_INVALID on any host."""
    from paper_1204_0069_gb300 import ccg
    L = ccg.lib()
    cfg = ccg.Config()
    L.ccg_config_init(ctypes.byref(cfg))
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert L.ccg_create(ctypes.byref(h), ctypes.byref(cfg)) == -1
    assert not h.value


def test_explicit_residual_needs_fp64(libpath):
    from paper_1204_0069_gb300 import ccg
    L = ccg.lib()
    cfg = ccg.Config()
    L.ccg_config_init(ctypes.byref(cfg))
    cfg.explicit_residual = 1
    cfg.precision = ccg.FP64_SLICED
    h = ctypes.c_void_p()
    assert L.ccg_create(ctypes.byref(h), ctypes.byref(cfg)) == -1


def test_invalid_arguments_rejected_before_any_device_work(libpath):
    from paper_1204_0069_gb300 import ccg
    L = ccg.lib()
    r = ccg.Result()
    # NULL handle -> CCG_ERR_INVALID without touching CUDA
    assert L.ccg_solve(None, 4, None, 4, None, None, 1, 1e-8, 10, None, ctypes.byref(r)) == -1
    assert L.ccg_destroy(None) == 0
    assert L.ccg_create(None, None) == -1


@pytest.mark.parametrize("field,value", [
    ("workers", 0), ("workers", 65), ("budget_bytes", 0.0), ("ctas_per_worker", -1),
    ("precision", 7), ("slots", -1), ("max_n", -1), ("max_p", -1), ("max_p", 33)])
def test_server_rejects_each_invalid_field_before_cuda(libpath, field, value):
    """ccg_server_create checks every field that does not depend on the
    device before its first CUDA call (CCG_ERR_INVALID on any host)."""
    from paper_1204_0069_gb300 import ccg
    L = ccg.lib()
    cfg = ccg.ServerConfig()
    L.ccg_server_config_init(ctypes.byref(cfg))
    setattr(cfg, field, value)
    srv = ctypes.c_void_p()
    assert L.ccg_server_create(ctypes.byref(cfg), ctypes.byref(srv)) == -1
    assert not srv.value


def test_server_slots_serve_fp64_only(libpath):
    from paper_1204_0069_gb300 import ccg
    L = ccg.lib()
    cfg = ccg.ServerConfig()
    L.ccg_server_config_init(ctypes.byref(cfg))
    cfg.slots = 8
    cfg.precision = ccg.FP8_IR
    srv = ctypes.c_void_p()
    assert L.ccg_server_create(ctypes.byref(cfg), ctypes.byref(srv)) == -1
