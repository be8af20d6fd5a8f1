"""Torch-facing wrapper of the CNN cell (argument marshalling only).

`Net` holds a libcloth network handle and its device workspace.
`CellFunction` exposes the cell to torch.autograd: its forward and backward
are libcloth's hand-written kernels (net_forward / net_backward).
Tensors are float32 CUDA: z (N, 6, H, W) = [u; v] with u = x - X, a (N, 3, H, W),
the weight blob (13036,) of which the first 13027 entries are trainable.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .cloth import _ptr, _require_cuda, _stream_handle

FP32, BF16 = _lib.NET_FP32, _lib.NET_BF16
N_PARAMS, N_BLOB = _lib.NET_PARAMS, _lib.NET_BLOB


class Net:
    def __init__(self, blob, precision: int = FP32, device="cuda", stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("Net needs a CUDA device (libcloth has no CPU path)")
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.precision = int(precision)
        self.stream = stream
        hb = np.ascontiguousarray(np.asarray(blob, dtype=np.float32))
        if hb.shape != (N_BLOB,):
            raise ValueError(f"weight blob must hold {N_BLOB} floats")
        n = ctypes.c_size_t()
        _lib.call("net_workspace_size", ctypes.byref(n))
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(n.value, dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            _lib.call("net_create", ctypes.byref(h), self.precision, hb.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                      _ptr(self.workspace), n.value, _stream_handle(stream))
        self.handle = h

    def _s(self):
        return _stream_handle(self.stream)

    def set_weights(self, w: torch.Tensor) -> None:
        _require_cuda(w, "weights")
        if w.numel() != N_BLOB:
            raise ValueError("weights must hold 13036 floats")
        _lib.call("net_set_weights", self.handle, _ptr(w), self._s())

    def get_weights(self) -> torch.Tensor:
        w = torch.empty(N_BLOB, dtype=torch.float32, device=self.device)
        _lib.call("net_get_weights", self.handle, _ptr(w), self._s())
        return w

    @staticmethod
    def saved_numel(N: int, H: int, W: int) -> int:
        n = ctypes.c_size_t()
        _lib.call("net_saved_size", int(N), int(H), int(W), ctypes.byref(n))
        return n.value // 4

    def forward(self, z: torch.Tensor, saved: torch.Tensor | None = None):
        """a = cell(z); returns (a, saved)."""
        _require_cuda(z, "z")
        N, C, H, W = z.shape
        if C != 6:
            raise ValueError("z must have 6 channels")
        a = torch.empty(N, 3, H, W, dtype=torch.float32, device=z.device)
        if saved is None and self.precision == FP32:
            saved = torch.empty(self.saved_numel(N, H, W), dtype=torch.float32, device=z.device)
        _lib.call("net_forward", self.handle, _ptr(z), _ptr(a), N, H, W, _ptr(saved), self._s())
        return a, saved

    def backward(self, z: torch.Tensor, saved: torch.Tensor, grad_a: torch.Tensor, grad_w: torch.Tensor | None = None,
                 need_grad_z: bool = True):
        """Adds dLoss/dw to grad_w (created zero if None); returns (grad_w, grad_z)."""
        _require_cuda(grad_a, "grad_a")
        N, _, H, W = z.shape
        if grad_w is None:
            grad_w = torch.zeros(N_PARAMS, dtype=torch.float32, device=z.device)
        gz = torch.empty_like(z) if need_grad_z else None
        _lib.call("net_backward", self.handle, _ptr(z), _ptr(saved), _ptr(grad_a.contiguous()), _ptr(gz), _ptr(grad_w),
                  N, H, W, self._s())
        return grad_w, gz

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.lib.net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adam_step(w: torch.Tensor, g: torch.Tensor, m: torch.Tensor, v: torch.Tensor, t: int, lr: float = 1e-3,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, n: int | None = None,
              mask: torch.Tensor | None = None) -> None:
    """One in-place Adam update of the first n entries of w (libcloth kernel);
    with `mask` (uint8 CUDA tensor of n bytes) only where it is non-zero."""
    n = int(n if n is not None else g.numel())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if mask is None:
        _lib.call("net_adam_step", _ptr(w), _ptr(g), _ptr(m), _ptr(v), n, int(t), ctypes.c_float(lr),
                  ctypes.c_float(beta1), ctypes.c_float(beta2), ctypes.c_float(eps), stream)
        return
    if not (mask.is_cuda and mask.dtype == torch.uint8 and mask.is_contiguous() and mask.numel() >= n):
        raise ValueError("mask must be a contiguous uint8 CUDA tensor of at least n entries")
    _lib.call("net_adam_step_masked", _ptr(w), _ptr(g), _ptr(m), _ptr(v), _ptr(mask), n, int(t), ctypes.c_float(lr),
              ctypes.c_float(beta1), ctypes.c_float(beta2), ctypes.c_float(eps), stream)


class CellFunction(torch.autograd.Function):
    """a = cell(z; w) with libcloth's forward and hand-written backward.

    Call as CellFunction.apply(z, w, net): w is the (13036,) blob tensor whose
    first 13027 entries receive gradients; the scales get zero gradient."""

    @staticmethod
    def forward(ctx, z, w, net: Net):
        net.set_weights(w.detach().contiguous())
        a, saved = net.forward(z.detach().contiguous())
        ctx.save_for_backward(z)
        ctx.saved_acts = saved
        ctx.net = net
        ctx.w = w
        return a

    @staticmethod
    def backward(ctx, grad_a):
        (z,) = ctx.saved_tensors
        net = ctx.net
        net.set_weights(ctx.w.detach().contiguous())
        gw, gz = net.backward(z.detach().contiguous(), ctx.saved_acts, grad_a.contiguous(), None,
                              need_grad_z=ctx.needs_input_grad[0])
        ctx.saved_acts = None
        full = torch.zeros(N_BLOB, dtype=torch.float32, device=gw.device)
        full[:N_PARAMS] = gw
        return gz, full, None
