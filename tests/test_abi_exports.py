"""The C ABI without a GPU: libmlsgd.so loads, exports every function that
include/mlsgd.h declares, the Python binding carries the same names, and the
host-only entry points behave as documented (no device call is made here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mlsgd.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return sorted(set(re.findall(r"\b(mlsgd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_09291_gb300 import build
    if not os.path.exists(build.LIB) or build._stale():
        if shutil.which(os.environ.get("NVCC", "nvcc")) is None:
            pytest.skip("nvcc not available and no built library")
        build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("mlsgd_create", "mlsgd_destroy", "mlsgd_sample_field", "mlsgd_solve_state_adjoint",
              "mlsgd_level_gradient", "mlsgd_step", "mlsgd_step_adaptive", "mlsgd_workspace_bytes",
              "mlsgd_solve_state_adjoint_noalloc"):
        assert n in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_uses_the_same_names():
    from paper_2606_09291_gb300 import mlsgd
    assert sorted(mlsgd.EXPORTS) == declared_functions()


def test_status_strings_and_argument_checks(lib):
    from paper_2606_09291_gb300 import mlsgd
    lib.mlsgd_status_string.argtypes = [ctypes.c_int]
    lib.mlsgd_status_string.restype = ctypes.c_char_p
    texts = [lib.mlsgd_status_string(s) for s in range(7)]
    assert all(t for t in texts) and len(set(texts)) == 7
    # configuration checks come before any device call: MLSGD_EINVAL (1)
    lib.mlsgd_create.argtypes = [ctypes.POINTER(mlsgd.Config), ctypes.POINTER(ctypes.c_void_p)]
    lib.mlsgd_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    assert lib.mlsgd_create(None, ctypes.byref(h)) == 1
    cfg = mlsgd.Config()
    cfg.n_levels, cfg.n0 = 0, 8  # no level
    assert lib.mlsgd_create(ctypes.byref(cfg), ctypes.byref(h)) == 1 and not h.value
    cfg.n_levels, cfg.n0 = 3, 6  # n0 not a power of two
    assert lib.mlsgd_create(ctypes.byref(cfg), ctypes.byref(h)) == 1 and not h.value
