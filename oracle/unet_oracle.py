"""CPU reference of the warm-start network (test infrastructure only).

Plain PyTorch on the CPU in float64: the same architecture as the GPU
network (two 3x3 convolutions + ReLU per encoder level, 2x2 average
pooling, nearest upsampling with additive skips, one 3x3 convolution per
decoder level, a linear 1x1 output), the masked mean-squared-error loss, and
parameter gradients by automatic differentiation.  Weights use the GPU
layout [Cout][9 Cin] with column t*Cin + c for tap t = 3 dy + dx, i.e. the
cross-correlation out[y][x] = sum w[dy][dx] in[y+dy-1][x+dx-1].
"""
import torch
import torch.nn.functional as F

CONVS = [("c0a", 8, 32), ("c0b", 32, 32), ("c1a", 32, 64), ("c1b", 64, 64), ("c2a", 64, 64), ("c2b", 64, 64),
         ("c3a", 64, 64), ("c3b", 64, 64), ("d2", 64, 64), ("d1", 64, 32), ("d0", 32, 32)]


def conv_weight(w, cin):
    """[Cout][9 Cin] (tap-major) -> conv2d weight [Cout][Cin][3][3]."""
    co = w.shape[0]
    return w.reshape(co, 9, cin).permute(0, 2, 1).reshape(co, cin, 3, 3)


def forward(params, x_nhwc, q=None):
    """params: name -> (w, b) float64 tensors (requires_grad as wanted);
    x_nhwc [B][S][S][8] -> prediction [B][S][S].

    q, if given, is applied to every activation the network stores between
    layers (the input, each convolution's output after ReLU, each pooled
    and each upsampled-plus-skip tensor; not the prediction): with q the
    rounding to the storage precision of an implementation, the result is
    that implementation's up to the order of its sums."""
    r = q if q is not None else (lambda t: t)
    x = r(x_nhwc).permute(0, 3, 1, 2)
    cin = dict((n, ci) for n, ci, _ in CONVS)

    def conv(name, t):
        w, b = params[name]
        return r(F.relu(F.conv2d(t, conv_weight(w, cin[name]), b, padding=1)))

    def pool(t):
        return r(F.avg_pool2d(t, 2))

    def up_add(t, skip):
        return r(F.interpolate(t, scale_factor=2, mode="nearest") + skip)

    s0 = conv("c0b", conv("c0a", x))
    s1 = conv("c1b", conv("c1a", pool(s0)))
    s2 = conv("c2b", conv("c2a", pool(s1)))
    b3 = conv("c3b", conv("c3a", pool(s2)))
    e2 = conv("d2", up_add(b3, s2))
    e1 = conv("d1", up_add(e2, s1))
    e0 = conv("d0", up_add(e1, s0))
    w, b = params["head"]
    return F.conv2d(e0, w.reshape(1, -1, 1, 1), b)[:, 0]


def masked_mse(pred, target, m):
    d = (pred - target)[:, :m, :m]
    return (d * d).sum() / (pred.shape[0] * m * m)
