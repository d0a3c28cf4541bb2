"""The C ABI library builds for sm_103a, loads without a GPU, exports every
function include/hjpdhg.h declares, and rejects bad arguments before touching
the device.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_1803_01215_gb300 import binding, build_lib

HEADER = os.path.join(build_lib.ROOT, "include", "hjpdhg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(hj_[a-z_0-9]+)\s*\(",
                                 src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(build_lib.lib_path()):
        build_lib.build()
    return ctypes.CDLL(build_lib.lib_path())


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("hj_problem_create", "hj_problem_destroy", "hj_solve_batch", "hj_status_str"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    for name in binding.EXPORTED:
        assert hasattr(lib, name), name


def test_status_strings_and_version(lib):
    lib.hj_status_str.restype = ctypes.c_char_p
    assert lib.hj_status_str(0) == b"ok"
    assert b"sigma" in lib.hj_status_str(3)
    assert lib.hj_version() >= 100


def test_invalid_arguments_rejected_before_device_use(lib):
    h = ctypes.c_void_p()
    W = (ctypes.c_double * 2)(1.0, 1.0)
    c = (ctypes.c_double * 2)(0.0, 0.0)
    assert lib.hj_problem_create(None, 0, 2, None, 0, W, c) == 1
    assert lib.hj_problem_create(ctypes.byref(h), 7, 2, None, 0, W, c) == 1       # family
    assert lib.hj_problem_create(ctypes.byref(h), 0, 0, None, 0, W, c) == 1       # d
    assert lib.hj_problem_create(ctypes.byref(h), 0, 129, None, 0, W, c) == 1     # d > 128
    assert lib.hj_problem_create(ctypes.byref(h), 1, 2, None, 0, W, c) == 1       # quadcopter d
    assert lib.hj_problem_create(ctypes.byref(h), 2, 2, None, 3, W, c) == 1       # A size
    nan = (ctypes.c_double * 2)(float("nan"), 1.0)
    assert lib.hj_problem_create(ctypes.byref(h), 0, 2, None, 0, nan, c) == 1
    opts = binding.make_opts(sigma=1.0, tau=0.24)
    lib.hj_solve_batch.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.POINTER(binding.SolverOpts)] + [ctypes.c_void_p] * 8
    assert lib.hj_solve_batch(None, 4, None, None, 8, ctypes.byref(opts),
                              None, None, None, None, None, None, None, None) == 1
    assert lib.hj_problem_destroy(None) == 0
