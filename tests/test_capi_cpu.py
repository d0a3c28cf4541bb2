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
                                   ctypes.POINTER(binding.SolverOpts)] + [ctypes.c_void_p] * 9
    assert lib.hj_solve_batch(None, 4, None, None, 8, ctypes.byref(opts),
                              None, None, None, None, None, None, None, None, None) == 1
    lib.hj_kkt_residual.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 4
    assert lib.hj_kkt_residual(None, 4, None, 8, 0, None, None, None, None) == 1
    lib.hj_shapes_save.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    lib.hj_shapes_load.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p]
    assert lib.hj_shapes_save(None, b"/tmp/x") == 1
    assert lib.hj_shapes_load(None, b"/tmp/x", None) == 1
    assert lib.hj_problem_destroy(None) == 0


def test_option_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of hj_solver_opts and hj_retry_policy have the C
    header's size and field offsets (a plain C probe compiled with the host
    compiler prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"hj_solver_opts": binding.SolverOpts, "hj_retry_policy": binding.RetryPolicy}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "hjpdhg.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
