"""Pins of the CPU reference network: the weight layout against a
brute-force loop convolution, pooling/upsampling against their definitions,
and the gradients against finite differences."""
import numpy as np
import torch

import oracle.unet_oracle as U


def test_conv_layout_matches_loop_definition():
    g = torch.Generator().manual_seed(0)
    B, S, ci, co = 1, 6, 3, 2
    x = torch.randn(B, S, S, ci, generator=g, dtype=torch.float64)
    w = torch.randn(co, 9 * ci, generator=g, dtype=torch.float64)
    b = torch.randn(co, generator=g, dtype=torch.float64)
    out = torch.nn.functional.conv2d(x.permute(0, 3, 1, 2), U.conv_weight(w, ci), b, padding=1)
    ref = np.zeros((B, co, S, S))
    xn, wn = x.numpy(), w.numpy()
    for o in range(co):
        for y in range(S):
            for xx in range(S):
                s = b[o].item()
                for t in range(9):
                    yy, xs = y + t // 3 - 1, xx + t % 3 - 1
                    if 0 <= yy < S and 0 <= xs < S:
                        for c in range(ci):
                            s += wn[o, t * ci + c] * xn[0, yy, xs, c]
                ref[0, o, y, xx] = s
    assert np.allclose(out.numpy(), ref, rtol=1e-12, atol=1e-12)


def test_network_gradients_match_finite_differences():
    g = torch.Generator().manual_seed(1)
    S, m = 16, 15
    params = {}
    for name, ci, co in U.CONVS:
        params[name] = (torch.randn(co, 9 * ci, generator=g, dtype=torch.float64) * (2.0 / (9 * ci)) ** 0.5,
                        torch.randn(co, generator=g, dtype=torch.float64) * 0.1)
    params["head"] = (torch.randn(1, 32, generator=g, dtype=torch.float64) * 0.3,
                      torch.zeros(1, dtype=torch.float64))
    x = torch.randn(1, S, S, 8, generator=g, dtype=torch.float64)
    tgt = torch.randn(1, S, S, generator=g, dtype=torch.float64)
    # directional derivatives d loss / d(param) . v by central differences
    # against automatic differentiation, a few random directions per tensor
    for name in ("c0a", "c2b", "c3a", "d1", "d0", "head"):
        w0, b0 = params[name]
        w = w0.clone().requires_grad_(True)
        b = b0.clone().requires_grad_(True)
        p = dict(params)
        p[name] = (w, b)
        U.masked_mse(U.forward(p, x), tgt, m).backward()
        for k in range(2):
            vw = torch.randn(w0.shape, generator=g, dtype=torch.float64)
            vb = torch.randn(b0.shape, generator=g, dtype=torch.float64)
            nv = float(torch.sqrt((vw * vw).sum() + (vb * vb).sum()))
            vw, vb = vw / nv, vb / nv          # unit direction: the step stays clear of ReLU kinks
            h = 1e-6

            def loss_at(t):
                q = dict(params)
                q[name] = (w0 + t * vw, b0 + t * vb)
                return float(U.masked_mse(U.forward(q, x), tgt, m))

            fd = (loss_at(h) - loss_at(-h)) / (2 * h)
            ad = float((w.grad * vw).sum() + (b.grad * vb).sum())
            assert abs(fd - ad) <= 1e-6 * max(1e-3, abs(ad)), (name, fd, ad)


def test_storage_rounding_hook_sees_every_stored_activation_in_order():
    """forward(..., q) applies q to the input and to every tensor the network
    stores between layers, in layer order: the 11 convolution outputs, the 3
    pooled and the 3 upsampled-plus-skip tensors (18 in all), never to the
    prediction; q = identity leaves the result unchanged, and with q the
    BF16 rounding each stored tensor is BF16-representable."""
    g = torch.Generator().manual_seed(2)
    S = 16
    params = {name: (torch.randn(co, 9 * ci, generator=g, dtype=torch.float64) * (2.0 / (9 * ci)) ** 0.5,
                     torch.randn(co, generator=g, dtype=torch.float64) * 0.1) for name, ci, co in U.CONVS}
    params["head"] = (torch.randn(1, 32, generator=g, dtype=torch.float64) * 0.3, torch.zeros(1, dtype=torch.float64))
    x = torch.randn(2, S, S, 8, generator=g, dtype=torch.float64)
    seen = []

    def record(t):
        seen.append(tuple(t.shape))
        return t

    base = U.forward(params, x)
    assert torch.equal(U.forward(params, x, q=record), base)
    # NHWC input, then NCHW activations: level-0 convs, pool, level-1 convs, ...
    expect = [(2, S, S, 8), (2, 32, S, S), (2, 32, S, S), (2, 32, S // 2, S // 2), (2, 64, S // 2, S // 2),
              (2, 64, S // 2, S // 2), (2, 64, S // 4, S // 4), (2, 64, S // 4, S // 4), (2, 64, S // 4, S // 4),
              (2, 64, S // 8, S // 8), (2, 64, S // 8, S // 8), (2, 64, S // 8, S // 8),
              (2, 64, S // 4, S // 4), (2, 64, S // 4, S // 4),      # up + skip, d2
              (2, 64, S // 2, S // 2), (2, 32, S // 2, S // 2),      # up + skip, d1
              (2, 32, S, S), (2, 32, S, S)]                          # up + skip, d0
    assert seen == expect

    def bf16(t):
        r = t.to(torch.bfloat16).to(torch.float64)
        seen.append(bool(torch.equal(r.to(torch.bfloat16).to(torch.float64), r)))
        return r

    seen.clear()
    rounded = U.forward(params, x, q=bf16)
    assert len(seen) == 18 and all(seen)
    # rounding every stored tensor to 8 significant bits moves the prediction
    # by a few tenths of a percent of its scale, not more
    assert 0 < float((rounded - base).abs().max()) <= 2e-2 * float(base.abs().max())
