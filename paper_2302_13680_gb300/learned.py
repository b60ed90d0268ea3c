"""Learned warm start: a small BF16 U-Net on the GPU kernels of libcmg.

The network maps two fields on the n x n grid -- the target state y_d and the
sample mean of log kappa_j -- to a control u0, used to start the multigrid
solve.  Every layer runs in libcmg's CUDA kernels (convolutions as im2col +
tcgen05 BF16 GEMM with FP32 accumulation, fused bias/ReLU; the backward pass
as split-K GEMMs and gather kernels; AdamW on FP32 master weights); this
module only allocates tensors and calls the C ABI in order.

Architecture (images padded to S x S, S = 256 for n = 255): four
resolutions 256/128/64/32 with 32, 64, 64, 64 channels, two 3x3
convolutions per encoder level, 2x2 average pooling, nearest upsampling with
additive skip connections, one 3x3 convolution per decoder level and a 1x1
output convolution.  Input channels: y_d, mean log kappa, 6 zero channels
(BF16 16-byte chunks hold 8 channels).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from .cmg import CMGError, load_library

CIN = 8
# name, input channels, output channels, resolution level
CONVS = [("c0a", CIN, 32, 0), ("c0b", 32, 32, 0),
         ("c1a", 32, 64, 1), ("c1b", 64, 64, 1),
         ("c2a", 64, 64, 2), ("c2b", 64, 64, 2),
         ("c3a", 64, 64, 3), ("c3b", 64, 64, 3),
         ("d2", 64, 64, 2), ("d1", 64, 32, 1), ("d0", 32, 32, 0)]
HEAD_C = 32


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@dataclass
class Param:
    w: object        # FP32 master [rows][cols]
    b: object        # FP32 [rows]
    w16: object      # BF16 copy used by the kernels
    mw: object
    vw: object
    mb: object
    vb: object
    gw: object = None
    gb: object = None


class WarmStartNet:
    def __init__(self, S: int = 256, batch: int = 8, seed: int = 0, device="cuda"):
        import torch

        if S % 8 or S < 16:
            raise ValueError("S must be a multiple of 8 and >= 16")
        self.S, self.B = S, batch
        self.dev = torch.device(device)
        self.lib = load_library()
        self._sig()
        g = torch.Generator().manual_seed(seed)
        self.params = {}
        for name, ci, co, _ in CONVS:
            std = math.sqrt(2.0 / (9 * ci))
            w = (torch.randn(co, 9 * ci, generator=g) * std)
            self.params[name] = self._param(w, torch.zeros(co))
        self.params["head"] = self._param(torch.randn(1, HEAD_C, generator=g) * 1e-2, torch.zeros(1))
        self.status = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self.step_count = 0
        self.in_scale = (1.0, 1.0)
        self.out_scale = 1.0

    # ---- C ABI signatures ------------------------------------------------
    def _sig(self):
        L = self.lib
        P, I, LL, D, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double, ctypes.c_float
        sig = {
            "cmg_nn_gemm_bf16": [P, LL, P, LL, I, I, I, P, I, P, P, I, P, P],
            "cmg_nn_gemm_bf16_splitk": [P, LL, P, LL, I, I, I, I, P, I, P, P],
            "cmg_nn_im2col": [P, P, I, I, I, I, I, P],
            "cmg_nn_col2im": [P, P, I, I, I, I, P],
            "cmg_nn_transpose": [P, P, LL, LL, P],
            "cmg_nn_relu_bwd": [P, P, P, LL, P],
            "cmg_nn_avgpool": [P, P, I, I, I, I, I, P],
            "cmg_nn_upsample_add": [P, P, P, I, I, I, I, P],
            "cmg_nn_upsample_bwd": [P, P, I, I, I, I, P],
            "cmg_nn_add": [P, P, P, LL, P],
            "cmg_nn_outer": [P, P, P, LL, I, P],
            "cmg_nn_to_bf16": [P, P, LL, P],
            "cmg_nn_sum_slices": [P, I, P, LL, P],
            "cmg_nn_colsum": [P, LL, I, P, P],
            "cmg_nn_mse": [P, P, I, I, I, P, P, I, ctypes.POINTER(I), P],
            "cmg_nn_adamw": [P, P, P, P, P, LL, F, F, F, F, F, I, P],
            "cmg_nn_pack_input": [P, P, I, I, I, I, F, F, P, P],
            "cmg_nn_unpack_output": [P, I, I, I, D, P, P],
            "cmg_nn_pack_target": [P, I, I, I, D, P, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.restype = ctypes.c_int
            fn.argtypes = args

    def _call(self, name, *args):
        st = getattr(self.lib, name)(*args)
        if st != 0:
            raise CMGError(st, name)

    def _param(self, w, b):
        import torch

        w = w.to(self.dev, torch.float32).contiguous()
        b = b.to(self.dev, torch.float32).contiguous()
        p = Param(w=w, b=b, w16=w.to(torch.bfloat16).contiguous(), mw=torch.zeros_like(w), vw=torch.zeros_like(w),
                  mb=torch.zeros_like(b), vb=torch.zeros_like(b))
        return p

    def refresh_bf16(self):
        for p in self.params.values():
            self._call("cmg_nn_to_bf16", _p(p.w), _p(p.w16), p.w.numel(), None)

    # ---- layers ------------------------------------------------------------
    def _res(self, level):
        return self.S >> level

    def _conv_fwd(self, name, X, B, H, ci, co):
        import torch

        P = B * H * H
        col = torch.empty(P, 9 * ci, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_im2col", _p(X), _p(col), B, H, H, ci, 0, None)
        Y = torch.empty(B, H, H, co, dtype=torch.bfloat16, device=self.dev)
        p = self.params[name]
        self._call("cmg_nn_gemm_bf16", _p(col), 9 * ci, _p(p.w16), 9 * ci, P, co, 9 * ci, _p(p.b), 1, None, _p(Y),
                   co, _p(self.status), None)
        return Y

    def _conv_bwd(self, name, X, Y, dY, B, H, ci, co, need_dx=True):
        import torch

        P = B * H * H
        p = self.params[name]
        dZ = torch.empty_like(Y)
        self._call("cmg_nn_relu_bwd", _p(Y), _p(dY), _p(dZ), Y.numel(), None)
        p.gb = torch.empty(co, dtype=torch.float32, device=self.dev)
        self._call("cmg_nn_colsum", _p(dZ), P, co, _p(p.gb), None)
        dZT = torch.empty(co, P, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_transpose", _p(dZ), _p(dZT), P, co, None)
        colT = torch.empty(9 * ci, P, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_im2col", _p(X), _p(colT), B, H, H, ci, 1, None)
        ks = min(4096, P)
        nsl = P // ks
        part = torch.empty(nsl, co, 9 * ci, dtype=torch.float32, device=self.dev)
        self._call("cmg_nn_gemm_bf16_splitk", _p(dZT), P, _p(colT), P, co, 9 * ci, ks, nsl, _p(part), 9 * ci,
                   _p(self.status), None)
        p.gw = torch.empty(co, 9 * ci, dtype=torch.float32, device=self.dev)
        self._call("cmg_nn_sum_slices", _p(part), nsl, _p(p.gw), co * 9 * ci, None)
        if not need_dx:
            return None
        WT = torch.empty(9 * ci, co, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_transpose", _p(p.w16), _p(WT), co, 9 * ci, None)
        dcol = torch.empty(P, 9 * ci, dtype=torch.float32, device=self.dev)
        self._call("cmg_nn_gemm_bf16", _p(dZ), co, _p(WT), co, P, 9 * ci, co, None, 0, _p(dcol), None, 9 * ci,
                   _p(self.status), None)
        dX = torch.empty(B, H, H, ci, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_col2im", _p(dcol), _p(dX), B, H, H, ci, None)
        return dX

    def _pool(self, X, B, H, C):
        import torch

        Y = torch.empty(B, H // 2, H // 2, C, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_avgpool", _p(X), _p(Y), B, H, H, C, 0, None)
        return Y

    def _pool_bwd(self, dY, B, H, C):
        import torch

        dX = torch.empty(B, H, H, C, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_avgpool", _p(dY), _p(dX), B, H, H, C, 1, None)
        return dX

    def _upadd(self, X, Ssk, B, H, C):
        import torch

        Y = torch.empty(B, H, H, C, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_upsample_add", _p(X), _p(Ssk), _p(Y), B, H, H, C, None)
        return Y

    def _up_bwd(self, dY, B, H, C):
        import torch

        dX = torch.empty(B, H, H, C, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_upsample_bwd", _p(dY), _p(dX), B, H, H, C, None)
        return dX

    def _add(self, a, b):
        import torch

        out = torch.empty_like(a)
        self._call("cmg_nn_add", _p(a), _p(b), _p(out), a.numel(), None)
        return out

    # ---- forward / backward ------------------------------------------------
    def forward(self, X):
        """X: [B][S][S][8] BF16 -> prediction [B][S][S] FP32; keeps activations."""
        import torch

        B, S = X.shape[0], self.S
        a = {}
        a["x0"] = X
        a["a0"] = self._conv_fwd("c0a", X, B, S, CIN, 32)
        a["s0"] = self._conv_fwd("c0b", a["a0"], B, S, 32, 32)
        a["p1"] = self._pool(a["s0"], B, S, 32)
        a["a1"] = self._conv_fwd("c1a", a["p1"], B, S // 2, 32, 64)
        a["s1"] = self._conv_fwd("c1b", a["a1"], B, S // 2, 64, 64)
        a["p2"] = self._pool(a["s1"], B, S // 2, 64)
        a["a2"] = self._conv_fwd("c2a", a["p2"], B, S // 4, 64, 64)
        a["s2"] = self._conv_fwd("c2b", a["a2"], B, S // 4, 64, 64)
        a["p3"] = self._pool(a["s2"], B, S // 4, 64)
        a["a3"] = self._conv_fwd("c3a", a["p3"], B, S // 8, 64, 64)
        a["b3"] = self._conv_fwd("c3b", a["a3"], B, S // 8, 64, 64)
        a["t2"] = self._upadd(a["b3"], a["s2"], B, S // 4, 64)
        a["e2"] = self._conv_fwd("d2", a["t2"], B, S // 4, 64, 64)
        a["t1"] = self._upadd(a["e2"], a["s1"], B, S // 2, 64)
        a["e1"] = self._conv_fwd("d1", a["t1"], B, S // 2, 64, 32)
        a["t0"] = self._upadd(a["e1"], a["s0"], B, S, 32)
        a["e0"] = self._conv_fwd("d0", a["t0"], B, S, 32, 32)
        pred = torch.empty(B, S, S, dtype=torch.float32, device=self.dev)
        h = self.params["head"]
        self._call("cmg_nn_gemm_bf16", _p(a["e0"]), HEAD_C, _p(h.w16), HEAD_C, B * S * S, 1, HEAD_C, _p(h.b), 0,
                   _p(pred), None, 1, _p(self.status), None)
        self._acts = a
        return pred

    def backward(self, dpred):
        """dpred: [B][S][S] BF16 gradient of the loss; fills every Param's gw, gb."""
        import torch

        a = self._acts
        B, S = a["x0"].shape[0], self.S
        P0 = B * S * S
        h = self.params["head"]
        e0T = torch.empty(HEAD_C, P0, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_transpose", _p(a["e0"]), _p(e0T), P0, HEAD_C, None)
        ks = min(4096, P0)
        nsl = P0 // ks
        part = torch.empty(nsl, 1, HEAD_C, dtype=torch.float32, device=self.dev)
        self._call("cmg_nn_gemm_bf16_splitk", _p(dpred), P0, _p(e0T), P0, 1, HEAD_C, ks, nsl, _p(part), HEAD_C,
                   _p(self.status), None)
        h.gw = torch.empty(1, HEAD_C, dtype=torch.float32, device=self.dev)
        self._call("cmg_nn_sum_slices", _p(part), nsl, _p(h.gw), HEAD_C, None)
        h.gb = torch.empty(1, dtype=torch.float32, device=self.dev)
        self._call("cmg_nn_colsum", _p(dpred), P0, 1, _p(h.gb), None)
        de0 = torch.empty(B, S, S, HEAD_C, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_outer", _p(dpred), _p(h.w), _p(de0), P0, HEAD_C, None)

        dt0 = self._conv_bwd("d0", a["t0"], a["e0"], de0, B, S, 32, 32)
        de1 = self._up_bwd(dt0, B, S // 2, 32)
        dt1 = self._conv_bwd("d1", a["t1"], a["e1"], de1, B, S // 2, 64, 32)
        de2 = self._up_bwd(dt1, B, S // 4, 64)
        dt2 = self._conv_bwd("d2", a["t2"], a["e2"], de2, B, S // 4, 64, 64)
        db3 = self._up_bwd(dt2, B, S // 8, 64)
        da3 = self._conv_bwd("c3b", a["a3"], a["b3"], db3, B, S // 8, 64, 64)
        dp3 = self._conv_bwd("c3a", a["p3"], a["a3"], da3, B, S // 8, 64, 64)
        ds2 = self._add(self._pool_bwd(dp3, B, S // 4, 64), dt2)
        da2 = self._conv_bwd("c2b", a["a2"], a["s2"], ds2, B, S // 4, 64, 64)
        dp2 = self._conv_bwd("c2a", a["p2"], a["a2"], da2, B, S // 4, 64, 64)
        ds1 = self._add(self._pool_bwd(dp2, B, S // 2, 64), dt1)
        da1 = self._conv_bwd("c1b", a["a1"], a["s1"], ds1, B, S // 2, 64, 64)
        dp1 = self._conv_bwd("c1a", a["p1"], a["a1"], da1, B, S // 2, 32, 64)
        ds0 = self._add(self._pool_bwd(dp1, B, S, 32), dt0)
        da0 = self._conv_bwd("c0b", a["a0"], a["s0"], ds0, B, S, 32, 32)
        self._conv_bwd("c0a", a["x0"], a["a0"], da0, B, S, CIN, 32, need_dx=False)

    def loss_and_grad(self, pred, target, m):
        """Masked MSE over the interior m x m region; returns (loss tensor, BF16 gradient)."""
        import torch

        B, S = pred.shape[0], self.S
        grad = torch.empty(B, S, S, dtype=torch.bfloat16, device=self.dev)
        cap = 152 * 32
        partial = torch.empty(cap, dtype=torch.float32, device=self.dev)
        used = ctypes.c_int()
        self._call("cmg_nn_mse", _p(pred), _p(target), B, S, m, _p(grad), _p(partial), cap, ctypes.byref(used), None)
        loss = partial[: used.value].double().sum() / (B * m * m)
        return loss, grad

    def adamw_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
        self.step_count += 1
        for p in self.params.values():
            self._call("cmg_nn_adamw", _p(p.w), _p(p.gw), _p(p.mw), _p(p.vw), _p(p.w16), p.w.numel(), lr, b1, b2,
                       eps, wd, self.step_count, None)
            self._call("cmg_nn_adamw", _p(p.b), _p(p.gb), _p(p.mb), _p(p.vb), None, p.b.numel(), lr, b1, b2, eps,
                       0.0, self.step_count, None)

    def check_status(self):
        if int(self.status.item()) != 0:
            raise CMGError(6, "a tensor-core completion wait exceeded its limit")

    # ---- data conversion ------------------------------------------------------
    def pack_inputs(self, yd, mlk, n):
        """yd, mlk: [B][n*n] FP64 CUDA -> [B][S][S][8] BF16 network input."""
        import torch

        B = yd.shape[0]
        X = torch.empty(B, self.S, self.S, CIN, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_nn_pack_input", _p(yd), _p(mlk), B, n, self.S, CIN, float(self.in_scale[0]),
                   float(self.in_scale[1]), _p(X), None)
        return X

    def pack_targets(self, u, n):
        import torch

        B = u.shape[0]
        T = torch.empty(B, self.S, self.S, dtype=torch.float32, device=self.dev)
        self._call("cmg_nn_pack_target", _p(u), B, n, self.S, 1.0 / self.out_scale, _p(T), None)
        return T

    def unpack(self, pred, n):
        import torch

        B = pred.shape[0]
        out = torch.empty(B, n * n, dtype=torch.float64, device=self.dev)
        self._call("cmg_nn_unpack_output", _p(pred), B, n, self.S, float(self.out_scale), _p(out), None)
        return out

    def state_dict(self):
        return {k: (p.w.cpu().numpy(), p.b.cpu().numpy()) for k, p in self.params.items()} | {
            "scales": (np.array(self.in_scale), np.array([self.out_scale]))}
