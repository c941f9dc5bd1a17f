"""The C-ABI library loads and exports every entry point include/ibm.h declares.

CPU only: the library is built if it is missing (nvcc cross-compiles for
sm_103a without a GPU) and opened with ctypes; no CUDA call is made.
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ibm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|size_t|const char\s*\*)\s*(ibm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_19920_gb300 import build
    path = build.LIB
    if not os.path.exists(path):
        build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary_entry_points():
    names = declared_functions()
    for required in ("ibm_plan_create", "ibm_plan_destroy", "ibm_poisson_solve", "ibm_helmholtz_solve",
                     "ibm_interp", "ibm_spread", "ibm_substep", "ibm_submit", "ibm_poll", "ibm_last_error",
                     "ibm_batch_create", "ibm_batch_poisson", "ibm_server_create"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_strings_without_gpu(lib):
    lib.ibm_version.restype = ctypes.c_char_p
    lib.ibm_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.ibm_version()
    # argument validation runs before any CUDA call
    out = ctypes.c_void_p()
    h = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    assert lib.ibm_plan_create(30, 32, 32, 1, h, 1, 1, ctypes.byref(out)) == -1
    assert b"nx=30" in lib.ibm_last_error()
    assert lib.ibm_plan_create(32, 32, 32, 7, h, 1, 1, ctypes.byref(out)) == -6


def test_noalloc_argument_checks_without_gpu(lib):
    """ibm_poisson_solve_noalloc validates its arguments, and rejects a grid
    larger than its static scratch with the bytes it would need, before any
    CUDA call; the optional status pointer does not take part in them."""
    lib.ibm_last_error.restype = ctypes.c_char_p
    f = lib.ibm_poisson_solve_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]
    h = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    a, b = 4096, 8192        # aligned stand-ins: never dereferenced, every call fails first
    status = ctypes.c_int(7)
    assert f(256, 256, 256, h, 1, a, b, ctypes.byref(status), None) == -1
    assert b"scratch" in lib.ibm_last_error()
    assert f(32, 32, 32, h, 1, a, a, ctypes.byref(status), None) == -1       # rhs == phi
    assert b"distinct" in lib.ibm_last_error()
    assert f(32, 32, 32, h, 1, a + 4, b, None, None) == -1                    # misaligned rhs
    assert b"aligned" in lib.ibm_last_error()
    assert f(30, 32, 32, h, 1, a, b, None, None) == -1
    assert f(32, 32, 32, h, 5, a, b, None, None) == -1
    assert f(32, 32, 32, None, 1, a, b, None, None) == -1
    assert status.value == 7  # untouched by calls that fail validation
