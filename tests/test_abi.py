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
