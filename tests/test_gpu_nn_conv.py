"""3x3 convolution as an implicit GEMM (cmg_nn_conv3x3_bf16: the tensor cores
read the NHWC activations through a TMA im2col map) against im2col + GEMM
through the C ABI (the same bits) and against an FP32 CPU convolution.

Shapes: the network's layers (8, 32 and 64 input channels; 32 and 64
outputs), 16, 24, 96 and 128 input channels, images whose pixel count is not a multiple of the 128-row tile
(the last tile runs past the last image), non-square images, an output
width that is not a multiple of 8 (scalar stores), and the first layer at
full size."""
import ctypes

import pytest
import torch
import torch.nn.functional as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    L = P.load_library()
    L.cmg_nn_conv3x3_bf16.restype = ctypes.c_int
    L.cmg_nn_conv3x3_bf16.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 4 + [ctypes.c_void_p, ctypes.c_int,
                                                                               ctypes.c_void_p, ctypes.c_int,
                                                                               ctypes.c_void_p, ctypes.c_void_p,
                                                                               ctypes.c_void_p]
    L.cmg_nn_im2col.restype = ctypes.c_int
    L.cmg_nn_im2col.argtypes = [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 5 + [ctypes.c_void_p]
    L.cmg_nn_gemm_bf16.restype = ctypes.c_int
    L.cmg_nn_gemm_bf16.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_longlong,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return L


def ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def data(B, H, W, C, Cout, seed):
    g = torch.Generator().manual_seed(seed)
    X = torch.randn(B, H, W, C, generator=g).to(torch.bfloat16)
    Wt = (torch.randn(Cout, 9 * C, generator=g) / (3 * C ** 0.5)).to(torch.bfloat16)
    bias = torch.randn(Cout, generator=g) * 0.1
    return X, Wt, bias


def cpu_conv(X, Wt, bias, relu):
    B, H, W, C = X.shape
    Cout = Wt.shape[0]
    w4 = Wt.float().view(Cout, 3, 3, C).permute(0, 3, 1, 2)          # column (3 dy + dx) C + c
    y = F.conv2d(X.float().permute(0, 3, 1, 2), w4, bias=bias, padding=1)
    y = y.permute(0, 2, 3, 1).reshape(B * H * W, Cout)
    return torch.relu(y) if relu else y


@pytest.mark.parametrize("B,H,W,C,Cout", [(2, 64, 64, 8, 32), (1, 32, 32, 32, 64), (2, 16, 16, 64, 64),
                                          (1, 4, 4, 64, 32), (3, 8, 12, 16, 40), (5, 8, 8, 8, 32),
                                          (2, 12, 20, 128, 48), (1, 6, 10, 96, 24), (1, 256, 256, 8, 32),
                                          (2, 128, 128, 32, 64), (2, 128, 128, 64, 64), (1, 8, 8, 24, 64)])
@pytest.mark.parametrize("relu", [0, 1])
def test_implicit_conv_equals_im2col_gemm_and_cpu(lib, B, H, W, C, Cout, relu):
    X, Wt, bias = data(B, H, W, C, Cout, seed=B * 1000 + H * 10 + C + Cout)
    P = B * H * W
    Xd, Wd, bd = X.cuda(), Wt.cuda(), bias.cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    Y = torch.full((P, Cout), float("nan"), dtype=torch.bfloat16, device="cuda")
    assert lib.cmg_nn_conv3x3_bf16(ptr(Xd), B, H, W, C, ptr(Wd), Cout, ptr(bd), relu, ptr(Y), ptr(status), s) == 0
    col = torch.empty(P, 9 * C, dtype=torch.bfloat16, device="cuda")
    Y2 = torch.full((P, Cout), float("nan"), dtype=torch.bfloat16, device="cuda")
    assert lib.cmg_nn_im2col(ptr(Xd), ptr(col), B, H, W, C, 0, s) == 0
    assert lib.cmg_nn_gemm_bf16(ptr(col), 9 * C, ptr(Wd), 9 * C, P, Cout, 9 * C, ptr(bd), relu, None, ptr(Y2), Cout,
                                ptr(status), s) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    # the same products summed in the same order: the same bits
    assert torch.equal(Y, Y2)
    # against the convolution on the CPU (FP32 from the same BF16 inputs; the
    # GPU output is rounded to BF16, 2^-8 relative)
    ref = cpu_conv(X, Wt, bias, relu)
    err = (Y.float().cpu() - ref).abs().max().item()
    assert err <= 8e-3 * ref.abs().max().item() + 1e-6, err


def test_implicit_conv_refuses_what_it_does_not_cover(lib, monkeypatch):
    X, Wt, bias = data(1, 8, 8, 8, 32, seed=1)
    Xd, Wd = X.cuda(), Wt.cuda()
    Y = torch.zeros(64, 65, dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    X4 = torch.zeros(1, 8, 8, 4, dtype=torch.bfloat16, device="cuda")
    W4 = torch.zeros(32, 36, dtype=torch.bfloat16, device="cuda")
    assert lib.cmg_nn_conv3x3_bf16(ptr(X4), 1, 8, 8, 4, ptr(W4), 32, None, 0, ptr(Y), ptr(status), s) == 7   # C % 8
    X40 = torch.zeros(1, 8, 8, 40, dtype=torch.bfloat16, device="cuda")
    W40 = torch.zeros(32, 360, dtype=torch.bfloat16, device="cuda")
    assert lib.cmg_nn_conv3x3_bf16(ptr(X40), 1, 8, 8, 40, ptr(W40), 32, None, 0, ptr(Y), ptr(status), s) == 7  # C = 40
    W65 = torch.zeros(65, 72, dtype=torch.bfloat16, device="cuda")
    assert lib.cmg_nn_conv3x3_bf16(ptr(Xd), 1, 8, 8, 8, ptr(W65), 65, None, 0, ptr(Y), ptr(status), s) == 7  # Cout
    assert lib.cmg_nn_conv3x3_bf16(None, 1, 8, 8, 8, ptr(Wd), 32, None, 0, ptr(Y), ptr(status), s) == 1
    monkeypatch.setenv("CMG_GEMM_TMA", "0")
    assert lib.cmg_nn_conv3x3_bf16(ptr(Xd), 1, 8, 8, 8, ptr(Wd), 32, None, 0, ptr(Y), ptr(status), s) == 7
    torch.cuda.synchronize()
    assert int(status.item()) == 0
