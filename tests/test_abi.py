"""The C-ABI library builds, loads without a GPU, exports every symbol that
include/mgct.h declares, and rejects bad arguments on the host before any
CUDA call."""
import ctypes
import os
import re

import pytest

from paper_2103_10329_gb300 import build as B
from paper_2103_10329_gb300 import mgct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return mgct.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mgct.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mgct_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mgct_geometry_create", "mgct_project", "mgct_backproject", "mgct_precondition",
                     "mgct_restrict_volume", "mgct_restrict_sino", "mgct_prolong_add",
                     "mgct_landweber_step", "mgct_osemtr_pass", "mgct_multigrid_iteration"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(L):
    assert L.mgct_status_string(0) == b"ok"
    assert L.mgct_status_string(-2) == b"inconsistent or unsupported sizes"


def test_host_side_argument_checks(L):
    # bad sizes and NULL pointers are rejected before any CUDA call
    assert L.mgct_restrict_volume(3, None, None, None) == -2
    assert L.mgct_restrict_volume(8, None, None, None) == -1
    assert L.mgct_restrict_sino(2, 3, 4, None, None, None) == -2
    assert L.mgct_project(None, 0, 0, 1, 1, None, 0, None, 0, None, None, None) == -1
    assert L.mgct_backproject(None, 0, 0, 1, 1, None, 0, None, 0, None) == -1
    assert L.mgct_landweber_step(None, 0, None, None, None, 0, None, None, None) == -1
    bad = ctypes.c_void_p(16 * 1000 + 4)
    assert L.mgct_restrict_volume(8, bad, bad, None) == -4
    assert b"aligned" in L.mgct_last_error()
    h = ctypes.c_void_p()
    desc = mgct.GeomDesc(64, 96, 96, 0, 2, 2.0, 4.0, 0.02, None, None, None, 2)
    assert L.mgct_geometry_create(ctypes.byref(desc), ctypes.byref(h)) == -1
    assert L.mgct_workspace_bytes(None, 0, 0) == 0
    assert L.mgct_net_check(None, None) == -1
    L.mgct_check_bounded_wait.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    flag = ctypes.c_int(0)
    assert L.mgct_check_bounded_wait(0.0, ctypes.byref(flag), None) == -1
    assert L.mgct_check_bounded_wait(0.1, None, None) == -1
    L.mgct_measure_onchip_peaks.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    x = ctypes.c_double(0.0)
    assert L.mgct_measure_onchip_peaks(None, ctypes.byref(x), None) == -1
    assert L.mgct_measure_onchip_peaks(ctypes.byref(x), None, None) == -1
