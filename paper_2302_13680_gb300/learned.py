"""Learned warm start: ctypes binding of libcmg's network handle (cmg_unet_*).

The network (a small BF16 U-Net mapping (y_d, sample mean of log kappa_j)
to a control u0) lives in the library: its weights, AdamW state, activation
buffers, the order of its layers forward and backward, and its checkpoints
(include/cmg.h, "learned warm start: the network as one handle").  This
module only checks tensors and passes pointers; PyTorch supplies device
memory and the stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .cmg import CMGError, load_library

CIN = 8
# name, input channels, output channels, resolution level (layer order of the handle)
CONVS = [("c0a", CIN, 32, 0), ("c0b", 32, 32, 0),
         ("c1a", 32, 64, 1), ("c1b", 64, 64, 1),
         ("c2a", 64, 64, 2), ("c2b", 64, 64, 2),
         ("c3a", 64, 64, 3), ("c3b", 64, 64, 3),
         ("d2", 64, 64, 2), ("d1", 64, 32, 1), ("d0", 32, 32, 0)]
LAYERS = [c[0] for c in CONVS] + ["head"]
HEAD_C = 32
ARRAYS = {"w": 0, "b": 1, "gw": 2, "gb": 3, "mw": 4, "vw": 5, "mb": 6, "vb": 7, "w16": 8}


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _sig(lib):
    P, I, D, F, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_ulonglong
    sig = {
        "cmg_unet_create": ([I, I, U64, P, ctypes.POINTER(P)], I),
        "cmg_unet_destroy": ([P], None),
        "cmg_unet_last_error": ([P], ctypes.c_char_p),
        "cmg_unet_set_scales": ([P, F, F, D], I),
        "cmg_unet_get_scales": ([P, ctypes.POINTER(F), ctypes.POINTER(F), ctypes.POINTER(D)], I),
        "cmg_unet_pack_inputs": ([P, P, P, I, I, P], I),
        "cmg_unet_pack_targets": ([P, P, I, I, P], I),
        "cmg_unet_unpack": ([P, P, I, I, P], I),
        "cmg_unet_forward": ([P, P, I, P], I),
        "cmg_unet_loss": ([P, P, I, P], I),
        "cmg_unet_backward": ([P, P], I),
        "cmg_unet_step": ([P, F, F, F, F, F], I),
        "cmg_unet_num_params": ([P], I),
        "cmg_unet_steps_taken": ([P], I),
        "cmg_unet_param_shape": ([P, I, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "cmg_unet_get": ([P, I, I, P], I),
        "cmg_unet_set": ([P, I, I, P], I),
        "cmg_unet_status": ([P, ctypes.POINTER(I)], I),
        "cmg_unet_save": ([P, ctypes.c_char_p], I),
        "cmg_unet_load": ([P, ctypes.c_char_p], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


class WarmStartNet:
    """One network handle (cmg_unet_create) for images S x S and batches of
    at most `batch`, enqueueing on the current CUDA stream."""

    def __init__(self, S: int = 256, batch: int = 8, seed: int = 0, device="cuda"):
        import torch

        self.lib = load_library()
        _sig(self.lib)
        self.S, self.B = int(S), int(batch)
        self.dev = torch.device(device)
        self.stream = torch.cuda.current_stream(self.dev)
        h = ctypes.c_void_p()
        st = self.lib.cmg_unet_create(self.S, self.B, int(seed), ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.byref(h))
        if st != 0:
            raise CMGError(st, "cmg_unet_create failed")
        self._h = h
        self._loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self._x = None   # input of the last forward pass, kept alive until backward

    def close(self):
        if getattr(self, "_h", None):
            self.lib.cmg_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        st = getattr(self.lib, name)(self._h, *args)
        if st != 0:
            msg = self.lib.cmg_unet_last_error(self._h)
            raise CMGError(st, f"{name}: {msg.decode() if msg else ''}")

    # ---- scales ----------------------------------------------------------
    @property
    def in_scale(self):
        a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_double()
        self._call("cmg_unet_get_scales", ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return (a.value, b.value)

    @property
    def out_scale(self):
        a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_double()
        self._call("cmg_unet_get_scales", ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return c.value

    def set_scales(self, in_yd: float, in_logk: float, out: float):
        self._call("cmg_unet_set_scales", float(in_yd), float(in_logk), float(out))

    # ---- data ------------------------------------------------------------
    def _check(self, t, dtype, shape, name):
        import torch

        if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != dtype or not t.is_contiguous():
            raise TypeError(f"{name}: expected a contiguous CUDA {dtype} tensor")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")

    def pack_inputs(self, yd, mlk, n):
        """yd, mlk: [B][n*n] FP64 CUDA -> [B][S][S][8] BF16 network input."""
        import torch

        B = yd.shape[0]
        self._check(yd, torch.float64, (B, n * n), "yd")
        self._check(mlk, torch.float64, (B, n * n), "mlk")
        X = torch.empty(B, self.S, self.S, CIN, dtype=torch.bfloat16, device=self.dev)
        self._call("cmg_unet_pack_inputs", _p(yd), _p(mlk), B, n, _p(X))
        return X

    def pack_targets(self, u, n):
        import torch

        B = u.shape[0]
        self._check(u, torch.float64, (B, n * n), "u")
        T = torch.empty(B, self.S, self.S, dtype=torch.float32, device=self.dev)
        self._call("cmg_unet_pack_targets", _p(u), B, n, _p(T))
        return T

    def unpack(self, pred, n):
        import torch

        B = pred.shape[0]
        self._check(pred, torch.float32, (B, self.S, self.S), "pred")
        out = torch.empty(B, n * n, dtype=torch.float64, device=self.dev)
        self._call("cmg_unet_unpack", _p(pred), B, n, _p(out))
        return out

    # ---- training ----------------------------------------------------------
    def forward(self, X):
        """X: [B][S][S][8] BF16 -> prediction [B][S][S] FP32 (activations kept)."""
        import torch

        B = X.shape[0]
        self._check(X, torch.bfloat16, (B, self.S, self.S, CIN), "X")
        pred = torch.empty(B, self.S, self.S, dtype=torch.float32, device=self.dev)
        self._call("cmg_unet_forward", _p(X), B, _p(pred))
        self._x = X
        return pred

    def loss(self, target, m):
        """Masked MSE of the last prediction over the interior m x m pixels
        (a CUDA double tensor); keeps the gradient for backward()."""
        import torch

        self._check(target, torch.float32, (target.shape[0], self.S, self.S), "target")
        self._call("cmg_unet_loss", _p(target), int(m), _p(self._loss))
        return self._loss

    def backward(self, dpred=None):
        """Gradients of every layer for the last forward pass, from the loss
        gradient kept by loss() or from dpred [B][S][S] BF16."""
        self._call("cmg_unet_backward", _p(dpred))

    def adamw_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
        self._call("cmg_unet_step", float(lr), float(b1), float(b2), float(eps), float(wd))

    @property
    def step_count(self):
        return int(self.lib.cmg_unet_steps_taken(self._h))

    def check_status(self):
        s = ctypes.c_int()
        self._call("cmg_unet_status", ctypes.byref(s))
        if s.value != 0:
            raise CMGError(6, "a tensor-core completion wait exceeded its limit")

    # ---- parameters and checkpoints -------------------------------------------
    def shape(self, layer: str):
        r, c = ctypes.c_int(), ctypes.c_int()
        self._call("cmg_unet_param_shape", LAYERS.index(layer), ctypes.byref(r), ctypes.byref(c))
        return r.value, c.value

    def get(self, layer: str, which: str) -> np.ndarray:
        rows, cols = self.shape(layer)
        n = rows if which in ("b", "gb", "mb", "vb") else rows * cols
        out = np.empty(n, dtype=np.float32)
        self._call("cmg_unet_get", LAYERS.index(layer), ARRAYS[which], out.ctypes.data_as(ctypes.c_void_p))
        return out if which in ("b", "gb", "mb", "vb") else out.reshape(rows, cols)

    def set(self, layer: str, which: str, values):
        rows, cols = self.shape(layer)
        n = rows if which in ("b", "gb", "mb", "vb") else rows * cols
        a = np.ascontiguousarray(np.asarray(values, dtype=np.float32).reshape(n))
        self._call("cmg_unet_set", LAYERS.index(layer), ARRAYS[which], a.ctypes.data_as(ctypes.c_void_p))

    def save(self, path: str):
        self._call("cmg_unet_save", str(path).encode())

    def load(self, path: str):
        self._call("cmg_unet_load", str(path).encode())
