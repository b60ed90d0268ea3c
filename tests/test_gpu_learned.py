"""The warm-start network's forward pass and parameter gradients on the GPU
(tcgen05 GEMMs + layer kernels) against the CPU float64 reference with
automatic differentiation.

Tolerances follow from BF16: activations, data gradients and GEMM operands
are rounded to 8 significant bits (relative 2^-9 = 0.2 %) at each of ~12
layers forward and ~24 backward, with FP32 accumulation; the resulting
norm-wise errors stay within a few percent, so outputs are held to 3 % and
gradients to 6 % (relative Frobenius norms)."""
import numpy as np
import pytest
import torch

import oracle.unet_oracle as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def net():
    from paper_2302_13680_gb300 import build

    build.build()
    from paper_2302_13680_gb300.learned import WarmStartNet

    return WarmStartNet(S=32, batch=2, seed=3)


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_forward_and_gradients_match_cpu_reference(net):
    g = torch.Generator().manual_seed(1)
    B, S, m = 2, 32, 31
    X = torch.zeros(B, S, S, 8)
    X[..., :2] = torch.randn(B, S, S, 2, generator=g)
    X = X.to(torch.bfloat16)
    tgt = torch.randn(B, S, S, generator=g)
    # a head large enough that the loss gradient reaches every layer, drawn
    # from a seeded generator (not the process-wide CUDA one, whose state
    # depends on which tests ran before)
    hg = torch.Generator().manual_seed(7)
    with torch.no_grad():
        w = net.params["head"].w
        w.copy_(torch.randn(w.shape, generator=hg) * 0.2)
    net.refresh_bf16()
    pred = net.forward(X.cuda())
    torch.cuda.synchronize()
    params = {k: (p.w16.double().cpu().clone().requires_grad_(True), p.b.double().cpu().clone().requires_grad_(True))
              for k, p in net.params.items()}
    ref = U.forward(params, X.double())
    assert rel(pred.double().cpu(), ref.detach()) <= 3e-2
    loss, grad = net.loss_and_grad(pred, tgt.cuda(), m)
    net.backward(grad)
    torch.cuda.synchronize()
    net.check_status()
    ref_loss = U.masked_mse(ref, tgt.double(), m)
    assert abs(float(loss) - float(ref_loss.detach())) <= 3e-2 * float(ref_loss.detach())
    ref_loss.backward()
    for k, p in net.params.items():
        gw_ref, gb_ref = params[k][0].grad, params[k][1].grad
        assert rel(p.gw.double().cpu(), gw_ref) <= 6e-2, k
        assert rel(p.gb.double().cpu(), gb_ref) <= 6e-2, k


def test_training_steps_reduce_the_loss(net):
    """A few AdamW steps on a fixed batch lower the masked MSE."""
    g = torch.Generator().manual_seed(2)
    B, S, m = 2, 32, 31
    X = torch.zeros(B, S, S, 8)
    X[..., :2] = torch.randn(B, S, S, 2, generator=g)
    X = X.to(torch.bfloat16).cuda()
    tgt = (torch.sin(torch.arange(S) * 0.3)[None, :, None] * torch.ones(B, S, S)).cuda()
    losses = []
    for _ in range(30):
        pred = net.forward(X)
        loss, grad = net.loss_and_grad(pred, tgt, m)
        net.backward(grad)
        net.adamw_step(lr=3e-3)
        losses.append(float(loss))
    net.check_status()
    assert losses[-1] < 0.5 * losses[0], losses
