"""The tensor-core GEMM's bounded waits run out and the kernel returns an
error status instead of hanging, through the C ABI.

cmg_nn_set_wait_limit(1) gives every operand and accumulator wait of the
TMA GEMM one poll: the first wait whose copy or tensor-core operation has not
landed gives up, the CTA stops issuing work, drains what it has in flight
(those waits keep the default limit), frees its tensor memory and sets the
call's status word.  The test reads that status, restores the default limit
and checks that the same call on the same context then computes the right
product (the context is intact), and that the status word is left as the
failed call set it (never cleared by a later call).  A GEMM with many K steps
(64) and more tiles than SMs makes the one-poll wait run out for certain."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    L = P.load_library()
    L.cmg_nn_gemm_bf16.restype = ctypes.c_int
    L.cmg_nn_gemm_bf16.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_longlong,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.cmg_nn_set_wait_limit.restype = ctypes.c_int
    L.cmg_nn_set_wait_limit.argtypes = [ctypes.c_longlong]
    yield L
    L.cmg_nn_set_wait_limit(0)


def ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_exhausted_wait_sets_status_and_context_survives(lib, monkeypatch):
    monkeypatch.delenv("CMG_GEMM_TMA", raising=False)
    M, N, K = 8192, 256, 4096
    g = torch.Generator().manual_seed(3)
    A = (torch.randn(M, K, generator=g) / 8).to(torch.bfloat16).cuda()
    B = (torch.randn(N, K, generator=g) / 8).to(torch.bfloat16).cuda()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    C = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.cmg_nn_set_wait_limit(-1) == 1            # CMG_ERR_INVALID_ARG
    assert lib.cmg_nn_set_wait_limit(1) == 0
    try:
        assert lib.cmg_nn_gemm_bf16(ptr(A), K, ptr(B), K, M, N, K, None, 0, ptr(C), None, N, ptr(status), s) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 1
    finally:
        assert lib.cmg_nn_set_wait_limit(0) == 0
    # the same context, the default limit: the right product, and the status
    # word still holds the failed call's 1
    C.zero_()
    assert lib.cmg_nn_gemm_bf16(ptr(A), K, ptr(B), K, M, N, K, None, 0, ptr(C), None, N, ptr(status), s) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 1
    ok = torch.zeros(1, dtype=torch.int32, device="cuda")
    C2 = torch.zeros_like(C)
    assert lib.cmg_nn_gemm_bf16(ptr(A), K, ptr(B), K, M, N, K, None, 0, ptr(C2), None, N, ptr(ok), s) == 0
    torch.cuda.synchronize()
    assert int(ok.item()) == 0
    assert torch.equal(C, C2)
    ref = A.float() @ B.float().T
    err = (C - ref).abs().max().item()
    assert err <= 1e-3 * ref.abs().max().item(), err
