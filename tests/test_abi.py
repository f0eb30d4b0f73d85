"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point include/sense.h declares; host-only calls behave."""
import ctypes
import os
import re

import pytest

from paper_1807_11830_gb300 import build as sense_build
from paper_1807_11830_gb300 import sense

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sense_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    path = sense_build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_operator_calls():
    names = declared_entry_points()
    for required in ("sense_forward", "sense_adjoint", "sense_normal", "sense_cg_solve", "sense_plan_create",
                     "sense_plan_destroy", "sense_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(declared_entry_points()):
        assert hasattr(lib, name), "libsense.so does not export %s" % name


def test_binding_covers_every_declared_symbol():
    assert set(sense.EXPORTED) <= declared_entry_points() | {"sense_plan_workspace_bytes"}
    for name in declared_entry_points():
        assert (name in sense.EXPORTED or name.startswith("sense_queue") or name.startswith("sense_sched")
                or name.startswith("sense_testing")), name


def test_size_table_is_host_only(lib):
    lib.sense_size_supported.restype = ctypes.c_int
    for n in sense.SIZES:
        assert lib.sense_size_supported(n) == 1
    for n in range(0, 1025):
        assert lib.sense_size_supported(n) == (1 if n in sense.SIZES else 0), n


def test_null_arguments_rejected_without_device(lib):
    lib.sense_plan_create.restype = ctypes.c_int
    lib.sense_plan_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.sense_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    assert lib.sense_plan_create(None, 0, ctypes.byref(out)) == 1  # SENSE_EINVAL
    assert b"NULL" in lib.sense_last_error()
    bad = sense._Shape(100, 100, 4, 1, 10, 0)
    assert lib.sense_plan_create(ctypes.byref(bad), 0, ctypes.byref(out)) == 2  # unsupported size
    lib.sense_forward.restype = ctypes.c_int
    lib.sense_forward.argtypes = [ctypes.c_void_p] * 6
    assert lib.sense_forward(None, None, None, None, None, None) == 1


def test_built_for_sm_103a(lib):
    log = open(os.path.join(ROOT, "_build", "ptxas.log")).read()
    assert "sm_103a" in log


def test_noalloc_size_limit_checked_before_any_device_work(lib):
    """sense_adjoint_noalloc rejects shapes beyond its fixed scratch (2^21
    complex values) on the host, before any CUDA call, so no device is needed."""
    lib.sense_adjoint_noalloc.restype = ctypes.c_int
    lib.sense_adjoint_noalloc.argtypes = [ctypes.c_void_p] * 6
    lib.sense_last_error.restype = ctypes.c_char_p
    over = sense._Shape(256, 256, 32, 3, 128, 0)   # 3*32*128*256 = 3*2^20 > 2^21
    assert lib.sense_adjoint_noalloc(ctypes.byref(over), None, None, None, None, None) == 1
    assert b"exceeds" in lib.sense_last_error()
    at_limit = sense._Shape(256, 256, 32, 2, 128, 0)  # exactly 2^21: size accepted, NULL pointers rejected
    assert lib.sense_adjoint_noalloc(ctypes.byref(at_limit), None, None, None, None, None) == 1
    assert b"aligned" in lib.sense_last_error()
    bad_size = sense._Shape(100, 100, 2, 1, 10, 0)
    assert lib.sense_adjoint_noalloc(ctypes.byref(bad_size), None, None, None, None, None) == 2
