"""tcgen05 BF16 GEMM of the warm-start network against an FP32 CPU matmul.

Every case runs through both kernels: the TMA-fed warp-specialised one (the
default) and the cp.async one (CMG_GEMM_TMA=0)."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gemm():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    lib = P.load_library()
    fn = lib.cmg_nn_gemm_bf16
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                   ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn


@pytest.fixture(params=["tma", "cp_async"])
def path(request, monkeypatch):
    monkeypatch.setenv("CMG_GEMM_TMA", "1" if request.param == "tma" else "0")
    return request.param


def ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# (2560, 2048, 320) and (6600, 384, 136) select the 256- and 128-column
# tiles of the TMA kernel (N a multiple of the tile, at least one tile per
# SM; the latter with a ragged M and a K of two full steps plus 8); the last
# two give each persistent CTA three or four tiles, so both TMEM
# accumulators are reused
@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 128, 192), (200, 50, 128), (1024, 64, 640), (131, 96, 64),
                                   (300, 1, 32), (128, 288, 72), (2560, 2048, 320), (6600, 384, 136),
                                   (40000, 96, 72), (70000, 40, 64)])
@pytest.mark.parametrize("epilogue", ["plain", "bias_relu"])
def test_gemm_matches_cpu(gemm, path, M, N, K, epilogue):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g) if epilogue == "bias_relu" else None
    ref = A.float() @ B.float().T
    if bias is not None:
        ref = torch.relu(ref + bias)
    Ad, Bd = A.cuda(), B.cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    C16 = torch.zeros(M, N, dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    bd = bias.cuda() if bias is not None else None
    st = gemm(ptr(Ad), K, ptr(Bd), K, M, N, K, ptr(bd), 1 if bias is not None else 0, ptr(C), ptr(C16), N,
              ptr(status), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = C.cpu()
    scale = ref.abs().max().item()
    # FP32 sums of K exact BF16 products: error ~ K * 2^-24 * |terms|
    assert (got - ref).abs().max().item() <= 1e-5 * K ** 0.5 * scale + 1e-6
    assert (C16.float().cpu() - ref).abs().max().item() <= 8e-3 * scale


def test_gemm_rejects_bad_shapes(gemm, path):
    A = torch.zeros(128, 96, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128, 64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert gemm(ptr(A), 96, ptr(A), 96, 128, 64, 12, None, 0, ptr(C), None, 64, ptr(status), None) == 1   # K % 8


# Kslice = 200 is not a multiple of the K step of 64: each slice's last step
# must read zeros, not the next slice's columns
@pytest.mark.parametrize("M,N,S,Z", [(64, 288, 1024, 6), (96, 40, 200, 5)])
def test_gemm_splitk_matches_cpu(gemm, path, M, N, S, Z):
    import paper_2302_13680_gb300 as P

    lib = P.load_library()
    fn = lib.cmg_nn_gemm_bf16_splitk
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int,
                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_void_p]
    g = torch.Generator().manual_seed(9 + S)
    A = torch.randn(M, S * Z, generator=g).to(torch.bfloat16)
    B = torch.randn(N, S * Z, generator=g).to(torch.bfloat16)
    part = torch.zeros(Z, M, N, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert fn(ptr(A.cuda()), S * Z, ptr(B.cuda()), S * Z, M, N, S, Z, ptr(part), N, ptr(status), None) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    for z in range(Z):
        ref = A[:, z * S:(z + 1) * S].float() @ B[:, z * S:(z + 1) * S].float().T
        assert (part[z].cpu() - ref).abs().max().item() <= 1e-5 * S ** 0.5 * ref.abs().max().item()


def test_gemm_row_stride_wider_than_k(gemm, path):
    # A and B are column windows of wider matrices (lda, ldb > K); C has ldc > N
    M, N, K, lda, ldb, ldc = 520, 200, 136, 200, 152, 208
    g = torch.Generator().manual_seed(31)
    Aw = torch.randn(M, lda, generator=g).to(torch.bfloat16)
    Bw = torch.randn(N, ldb, generator=g).to(torch.bfloat16)
    ref = Aw[:, :K].float() @ Bw[:, :K].float().T
    C = torch.full((M, ldc), 7.0, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert gemm(ptr(Aw.cuda()), lda, ptr(Bw.cuda()), ldb, M, N, K, None, 0, ptr(C), None, ldc, ptr(status), None) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = C.cpu()
    assert (got[:, :N] - ref).abs().max().item() <= 1e-5 * K ** 0.5 * ref.abs().max().item() + 1e-6
    assert bool((got[:, N:] == 7.0).all())   # columns past N untouched


def test_wait_limit_gives_up_cleanly_and_the_next_call_runs(gemm, monkeypatch):
    """With the TMA kernel's work waits limited to one poll, a call gives up
    (status word set; the kernel drains what it has in flight and frees its
    tensor memory); with the default limit restored, the next call on the
    same stream is exact again."""
    import paper_2302_13680_gb300 as P

    monkeypatch.setenv("CMG_GEMM_TMA", "1")
    lib = P.load_library()
    setl = lib.cmg_nn_set_wait_limit
    setl.argtypes = [ctypes.c_longlong]
    setl.restype = ctypes.c_int
    g = torch.Generator().manual_seed(5)
    M, N, K = 4096, 256, 512
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    ref = A.float().cpu() @ B.float().cpu().T
    try:
        assert setl(1) == 0
        gave_up = False
        for _ in range(3):
            C = torch.zeros(M, N, device="cuda")
            status = torch.zeros(1, dtype=torch.int32, device="cuda")
            assert gemm(ptr(A), K, ptr(B), K, M, N, K, None, 0, ptr(C), None, N, ptr(status), None) == 0
            torch.cuda.synchronize()
            gave_up = gave_up or int(status.item()) == 1
        assert gave_up
    finally:
        assert setl(0) == 0
    C = torch.zeros(M, N, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert gemm(ptr(A), K, ptr(B), K, M, N, K, None, 0, ptr(C), None, N, ptr(status), None) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert float((C.cpu() - ref).abs().max()) <= 1e-3 * float(ref.abs().max())
    assert setl(-1) == 1   # refused
