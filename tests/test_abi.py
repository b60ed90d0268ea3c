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
    """Every problem below is rejected before any device call, each for its
    own defect (a valid xi is passed, so a missing one is not the reason)."""
    import numpy as np

    from paper_2302_13680_gb300 import cmg

    L = cmg.load_library()
    h = ctypes.c_void_p()
    xi = np.zeros((4096, 4))
    xp = xi.ctypes.data_as(ctypes.c_void_p)
    local = cmg._box((0.25, 0.75, 0.25, 0.75))
    for bad in [cmg.Problem(30, 8, 4, 1e-4, 0.5, 3, 0),      # n not 2^l - 1
                cmg.Problem(31, 0, 4, 1e-4, 0.5, 3, 0),      # N < 1
                cmg.Problem(31, 8, 4, -1.0, 0.5, 3, 0),      # nu <= 0
                cmg.Problem(31, 8, 4, 1e-4, 0.5, 5, 0),      # coarsest not 1, 3, 7
                cmg.Problem(3, 8, 4, 1e-4, 0.5, 7, 0),       # coarsest > n
                cmg.Problem(31, 8, 4, 1e-4, 0.5, 3, 3),      # unknown coarse-operator rule
                cmg.Problem(31, 8, 4, 1e-4, 0.5, 3, 0, cmg._box((0.5, 0.25, 0.0, 1.0))),   # control box x1 < x0
                cmg.Problem(31, 8, 4, 1e-4, 0.5, 3, 0, cmg._box((0.0, 1.5, 0.0, 1.0))),    # outside the square
                cmg.Problem(31, 8, 4, 1e-4, 0.5, 3, 0, cmg._box((0.2, 0.8, 0.3, float("nan"))))]:
        assert L.cmg_create(ctypes.byref(bad), xp, None, ctypes.byref(h)) == 1
    assert L.cmg_create(ctypes.byref(cmg.Problem(31, 8, 4, 1e-4, 0.5, 3, 0)), None, None,
                        ctypes.byref(h)) == 1        # K > 0 and no xi
    assert L.cmg_create(ctypes.byref(cmg.Problem(31, 4096, 4, 1e-4, 0.5, 3, 0)), xp, None,
                        ctypes.byref(h)) == 7        # N above the kernels' limit
    assert L.cmg_create(ctypes.byref(cmg.Problem(31, 8, 4, 1e-4, 0.5, 3, cmg.COARSE["galerkin"], local)), xp, None,
                        ctypes.byref(h)) == 7        # Galerkin operators with local control
    assert L.cmg_num_levels(None) == 0
    assert L.cmg_level_n(None, 0) == -1


def header_constants():
    text = open(os.path.join(ROOT, "include", "cmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    vals = {k: int(v) for k, v in re.findall(r"\b(CMG_\w+)\s*=\s*(-?\d+)", text)}
    vals.update({k: int(v) for k, v in re.findall(r"#define\s+(CMG_\w+)\s+(\d+)", text)})
    return vals


def test_binding_constants_match_the_header():
    from paper_2302_13680_gb300 import cmg

    c = header_constants()
    assert cmg.STATUS == {c["CMG_OK"]: "OK", c["CMG_ERR_INVALID_ARG"]: "INVALID_ARG", c["CMG_ERR_CUDA"]: "CUDA",
                          c["CMG_ERR_OOM"]: "OOM", c["CMG_ERR_NOT_CONVERGED"]: "NOT_CONVERGED",
                          c["CMG_ERR_NONFINITE"]: "NONFINITE", c["CMG_ERR_TIMEOUT"]: "TIMEOUT",
                          c["CMG_ERR_UNSUPPORTED"]: "UNSUPPORTED"}
    assert (cmg.SMOOTH_RBGS, cmg.SMOOTH_JACOBI) == (c["CMG_SMOOTH_RBGS"], c["CMG_SMOOTH_JACOBI"])
    assert (cmg.FP64, cmg.FP32) == (c["CMG_FP64"], c["CMG_FP32"])
    assert (cmg.METHOD_CYCLE, cmg.METHOD_FGMRES) == (c["CMG_METHOD_CYCLE"], c["CMG_METHOD_FGMRES"])
    assert cmg.COARSE == {"averaged": c["CMG_COARSE_AVERAGED"], "nodal": c["CMG_COARSE_NODAL"],
                          "galerkin": c["CMG_COARSE_GALERKIN"]}
    assert (cmg.KERNEL_SMOOTH, cmg.KERNEL_RESIDUAL, cmg.KERNEL_RESTRICT, cmg.KERNEL_PROLONG, cmg.KERNEL_COARSE,
            cmg.KERNEL_TAIL) == tuple(c["CMG_KERNEL_" + k] for k in ("SMOOTH", "RESIDUAL", "RESTRICT", "PROLONG",
                                                                       "COARSE", "TAIL"))
    assert (c["CMG_TUNE_STAGED"], c["CMG_TUNE_WIDE"]) == (16, 32)   # the flags the tests and tuning cache use
    assert c["CMG_TUNE_UNFUSED"] == 64 and c["CMG_TUNE_FUSED"] == 128
    assert (cmg.BATCH_AUTO, cmg.BATCH_PERSISTENT, cmg.BATCH_BRANCHES) == \
        (c["CMG_BATCH_AUTO"], c["CMG_BATCH_PERSISTENT"], c["CMG_BATCH_BRANCHES"])
    assert (cmg.BATCH_LEGS_BY_WORK, cmg.BATCH_LEGS_PERSISTENT, cmg.BATCH_LEGS_PHASES) == \
        (c["CMG_BATCH_LEGS_BY_WORK"], c["CMG_BATCH_LEGS_PERSISTENT"], c["CMG_BATCH_LEGS_PHASES"])


def test_sample_map_covers_every_sample_and_matches_the_stated_limits(lib):
    """The node kernels' launch shape (cmg_sample_map, host arithmetic):
    every sample of a node is covered by its lanes x chunks x vector width,
    lanes and chunks are powers of two, vectors divide N and fit 16 bytes;
    the wide FP32 layout takes 2 samples a lane; and the shapes the kernels
    cannot take are exactly the N the header excludes (N > 256 not a
    multiple of 4, N > 512), which cmg_create refuses before any device call."""
    import numpy as np

    from paper_2302_13680_gb300 import cmg

    L = cmg.load_library()
    fn = L.cmg_sample_map
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
    lpn, V, spl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    pow2 = {1, 2, 4, 8, 16, 32, 64, 128, 256, 512}
    for N in range(1, 521):
        for eb in (4, 8):
            for items in (0, 1, 961, 65025, 10 ** 6):
                for target in (0, 1, 2, 4, 16 | 1, 16 | 2, 32 | 1):
                    st = fn(N, eb, items, target, ctypes.byref(lpn), ctypes.byref(V), ctypes.byref(spl))
                    l, v, c = lpn.value, V.value, spl.value
                    assert l in pow2 and l <= 32 and c in pow2
                    assert v in (1, 2, 4) and v * eb <= 16 and N % v == 0
                    assert l * c * v >= N
                    if target & 32 and eb == 4 and N % 2 == 0 and N <= 64:
                        assert (v, c) == (2, 1) and 2 * l >= N
                    assert st == (0 if c <= 8 else 7)
        ok = all(fn(N, eb, 0, 0, ctypes.byref(lpn), ctypes.byref(V), ctypes.byref(spl)) == 0 for eb in (4, 8))
        assert ok == (N <= 256 or (N % 4 == 0 and N <= 512)), N
        if not ok:
            xi = np.zeros((N, 1))
            h = ctypes.c_void_p()
            assert L.cmg_create(ctypes.byref(cmg.Problem(31, N, 1, 1e-4, 0.5, 3, 0)), xi.ctypes.data_as(ctypes.c_void_p),
                                None, ctypes.byref(h)) == 7
    assert fn(0, 4, 0, 0, ctypes.byref(lpn), ctypes.byref(V), ctypes.byref(spl)) == 1
    assert fn(8, 2, 0, 0, ctypes.byref(lpn), ctypes.byref(V), ctypes.byref(spl)) == 1


def test_unet_create_rejects_bad_sizes_before_any_device_call(lib):
    """The network handle refuses image sides that are not multiples of 32,
    batch sizes outside [1, 1024] and a null output, with no GPU present."""
    create = lib.cmg_unet_create
    create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_void_p,
                       ctypes.POINTER(ctypes.c_void_p)]
    create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    for S, B in [(30, 2), (16, 2), (8192, 2), (64, 0), (64, 2000)]:
        assert create(S, B, 0, None, ctypes.byref(h)) == 1, (S, B)
        assert not h.value
    assert create(64, 2, 0, None, None) == 1


def test_unet_binding_constants_match_the_header():
    """learned.py's array codes and layer order equal include/cmg.h's."""
    from paper_2302_13680_gb300 import learned

    text = open(os.path.join(ROOT, "include", "cmg.h")).read()
    for name, code in learned.ARRAYS.items():
        m = re.search(rf"CMG_UNET_{name.upper()}\s*=\s*(\d+)", text)
        assert m and int(m.group(1)) == code, name
    order = re.search(r"Layers 0\.\.10 are the 3x3 convolutions (.*?) \(weights", text, flags=re.S).group(1)
    names = [w.strip(" ,*\n") for w in re.split(r"[,\s]+", order.replace("*", " ")) if w.strip(" ,*\n")]
    assert names == learned.LAYERS[:11], names
