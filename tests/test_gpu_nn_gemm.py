"""tcgen05 BF16 GEMM of the warm-start network against an FP32 CPU matmul."""
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


def ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 128, 192), (200, 50, 128), (1024, 64, 640), (131, 96, 64),
                                   (300, 1, 32), (128, 288, 72)])
@pytest.mark.parametrize("epilogue", ["plain", "bias_relu"])
def test_gemm_matches_cpu(gemm, M, N, K, epilogue):
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


def test_gemm_rejects_bad_shapes(gemm):
    A = torch.zeros(128, 96, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128, 64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert gemm(ptr(A), 96, ptr(A), 96, 128, 64, 12, None, 0, ptr(C), None, 64, ptr(status), None) == 1   # K % 8


def test_gemm_splitk_matches_cpu(gemm):
    import paper_2302_13680_gb300 as P

    lib = P.load_library()
    fn = lib.cmg_nn_gemm_bf16_splitk
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int,
                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_void_p]
    M, N, S, Z = 64, 288, 1024, 6
    g = torch.Generator().manual_seed(9)
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
