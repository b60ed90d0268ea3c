"""Host-side checks of the C ABI: the library builds for sm_103a, loads on a
machine without a GPU, and exports every function include/cmg.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(cmg_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2302_13680_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["cmg_create", "cmg_destroy", "cmg_set_samples", "cmg_residual", "cmg_smooth",
                     "cmg_restrict", "cmg_prolong_add", "cmg_coarse_solve", "cmg_cycle_apply", "cmg_solve",
                     "cmg_norm", "cmg_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_rejects_bad_sizes(lib):
    from paper_2302_13680_gb300 import cmg

    L = cmg.load_library()
    h = ctypes.c_void_p()
    for bad in [cmg.Problem(30, 8, 4, 1e-4, 0.5, 3, 0),      # n not 2^l - 1
                cmg.Problem(31, 0, 4, 1e-4, 0.5, 3, 0),      # N < 1
                cmg.Problem(31, 8, 4, -1.0, 0.5, 3, 0),      # nu <= 0
                cmg.Problem(31, 8, 4, 1e-4, 0.5, 5, 0),      # coarsest not 1, 3, 7
                cmg.Problem(3, 8, 4, 1e-4, 0.5, 7, 0),       # coarsest > n
                cmg.Problem(31, 8, 4, 1e-4, 0.5, 3, 2),      # unknown coarse-coefficient rule
                cmg.Problem(31, 8, 4, 1e-4, 0.5, 3, 0, cmg._box((0.5, 0.25, 0.0, 1.0))),   # control box x1 < x0
                cmg.Problem(31, 8, 4, 1e-4, 0.5, 3, 0, cmg._box((0.0, 1.5, 0.0, 1.0))),    # outside the square
                cmg.Problem(31, 8, 4, 1e-4, 0.5, 3, 0, cmg._box((0.2, 0.8, 0.3, float("nan"))))]:
        assert L.cmg_create(ctypes.byref(bad), None, None, ctypes.byref(h)) == 1
    assert L.cmg_create(ctypes.byref(cmg.Problem(31, 4096, 0, 1e-4, 0.5, 3, 0)), None, None,
                        ctypes.byref(h)) == 7        # N above the kernels' limit
    assert L.cmg_num_levels(None) == 0
    assert L.cmg_level_n(None, 0) == -1
