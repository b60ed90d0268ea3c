"""The allocation-free norm entry point against cmg_norm and against numpy, through
the C ABI.

cmg_norm_noalloc serves callers that cannot allocate device memory where
they need a norm (an embedding application that owns all allocations, or a
loop that must not allocate): it keeps its partial sums in a static device
array instead of handle memory.  This file is collected last so that a
failure here cannot hide any other test's result, and it passes both alone
in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def env():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    lib = P.load_library()
    fn = lib.cmg_norm_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_double,
                                           ctypes.c_void_p, ctypes.c_void_p]
    pr = inputs.make_problem(**inputs.CONFIGS["n31_N8"])
    H = P.Hierarchy(pr.n, pr.N, pr.xi, pr.nu, pr.amp)
    yield H, fn
    H.close()


def call(fn, v, wy, out, stream):
    y, u, p = v
    return fn(ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(p.data_ptr()),
              y.numel(), u.numel(), wy, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_norm_matches_cmg_norm_twice(env):
    H, fn = env
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    outs = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    vecs = []
    for k in range(2):
        v = tuple(torch.tensor(rng.standard_normal(t.shape) * (k + 1), device="cuda") for t in H.zeros(0))
        vecs.append(v)
        assert call(fn, v, 1.0, outs[k:k + 1], stream) == 0
    torch.cuda.synchronize()
    for k in range(2):
        ref = H.norm(0, vecs[k])
        got = float(outs[k].item())
        assert abs(got - ref) <= TOL64 * ref, (k, got, ref)
        # and against the norm computed on the host by numpy (FP64)
        host = float(np.sqrt(sum(np.sum(t.cpu().numpy() ** 2) for t in vecs[k])))
        assert abs(got - host) <= TOL64 * host, (k, got, host)
    # weighted form: the y segment scaled by wy
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert call(fn, vecs[0], float(H.N), out, stream) == 0
    torch.cuda.synchronize()
    scaled = (vecs[0][0] * H.N, vecs[0][1], vecs[0][2])
    ref = H.norm(0, scaled)
    assert abs(float(out.item()) - ref) <= TOL64 * ref
    host = float(np.sqrt(sum(np.sum(t.cpu().numpy() ** 2) for t in scaled)))
    assert abs(float(out.item()) - host) <= TOL64 * host


def test_noalloc_rejects_sizes_beyond_the_static_array(env):
    H, fn = env
    v = H.zeros(0)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    y, u, p = v
    st = fn(ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(p.data_ptr()),
            (1 << 28) + 1, u.numel(), 1.0, ctypes.c_void_p(out.data_ptr()), None)
    assert st == 7        # CMG_ERR_UNSUPPORTED, nothing enqueued
    st = fn(None, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(p.data_ptr()), 10, 10, 1.0,
            ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1        # CMG_ERR_INVALID_ARG
