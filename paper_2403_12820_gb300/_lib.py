"""ctypes binding of libcloth (include/cloth.h): argument marshalling only.

Every entry point keeps its C name.  The library is built in-tree on first
use (nvcc, sm_103a) if it is missing or stale; if it cannot be built or
loaded, loading fails loudly — there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int32, c_int64, c_float, c_size_t, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p
P = ctypes.POINTER

CLOTH_OK = 0
NET_FP32, NET_BF16 = 0, 1
NET_PARAMS, NET_BLOB = 13027, 13036
PCELL_BLOB = 40
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "ETIMEOUT", -6: "EUNSUPPORTED"}
STATUS_NONFINITE, STATUS_TIMEOUT, STATUS_BOUNDS = 1, 2, 4


class ClothGrid(ctypes.Structure):
    _fields_ = [("rows", c_int32), ("cols", c_int32), ("spacing", c_float), ("mass", c_float)]


class ClothParams(ctypes.Structure):
    _fields_ = [("k_struct", c_float), ("k_shear", c_float), ("k_bend", c_float), ("mu_spring", c_float),
                ("drag", c_float), ("pressure", c_float), ("gravity", c_float * 3)]


class ClothPins(ctypes.Structure):
    _fields_ = [("count", c_int32), ("node", P(c_int32)), ("velocity", c_float * 3)]


class ClothSphere(ctypes.Structure):
    _fields_ = [("center", c_float * 3), ("radius", c_float), ("enabled", c_int32), ("friction", c_float)]


class RolloutOpts(ctypes.Structure):
    _fields_ = [("steps", c_int32), ("graph_chunk", c_int32), ("d_record", c_void_p), ("record_every", c_int32)]


class NetRolloutOpts(ctypes.Structure):
    _fields_ = [("steps", c_int32), ("check_every", c_int32), ("residual_bound", c_float), ("graph_chunk", c_int32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "cloth_workspace_size": (c_int32, [c_int32, P(ClothGrid), P(c_size_t)]),
    "cloth_create": (c_int32, [P(c_void_p), c_int32, P(ClothGrid), P(ClothParams), P(ClothPins), P(ClothSphere),
                               c_float, c_void_p, c_size_t, c_void_p]),
    "cloth_set_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "cloth_get_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "cloth_forces": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "cloth_step_plain": (c_int32, [c_void_p, c_int32, c_void_p]),
    "cloth_rollout_plain": (c_int32, [c_void_p, P(RolloutOpts), c_void_p]),
    "cloth_topology": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p]),
    "cloth_set_launch": (c_int32, [c_void_p, c_int32, c_int32, c_void_p]),
    "cloth_get_launch": (c_int32, [c_void_p, P(c_int32), P(c_int32), P(c_int32)]),
    "cloth_net_tile_choices": (c_int32, [c_int32, P(c_int32), P(c_int32), P(c_int32), c_int32, P(c_int32)]),
    "cloth_set_net_tile": (c_int32, [c_void_p, c_int32, c_int32]),
    "cloth_get_net_tile": (c_int32, [c_void_p, c_int32, P(c_int32)]),
    "cloth_tune_net": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, P(c_float), P(c_int32), c_void_p,
                                 ctypes.c_size_t, c_void_p]),
    "cloth_set_boundary": (c_int32, [c_void_p, c_int32, P(c_float), c_float, c_void_p]),
    "cloth_set_net_stride": (c_int32, [c_void_p, c_int32, c_void_p]),
    "cloth_set_train_segment": (c_int32, [c_void_p, c_int32]),
    "cloth_selftest_wait_timeout": (c_int32, [c_void_p, c_int32, c_void_p]),
    "cloth_implicit_workspace_size": (c_int32, [c_void_p, P(c_size_t)]),
    "cloth_step_implicit": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_size_t, c_void_p]),
    "cloth_tune_launch": (c_int32, [c_void_p, c_int32, P(c_int32), P(c_int32), c_int32, c_int32, P(c_float),
                                    P(c_int32), c_void_p]),
    "cloth_status": (c_int32, [c_void_p, P(c_int32), c_int32, c_void_p]),
    "net_workspace_size": (c_int32, [P(c_size_t)]),
    "net_create": (c_int32, [P(c_void_p), c_int32, P(c_float), c_void_p, c_size_t, c_void_p]),
    "net_set_weights": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "net_get_weights": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "net_saved_size": (c_int32, [c_int32, c_int32, c_int32, P(c_size_t)]),
    "net_forward": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p]),
    "net_backward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32,
                               c_void_p]),
    "net_destroy": (None, [c_void_p]),
    "net_forward_static": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_void_p]),
    "cloth_net_workspace_size": (c_int32, [c_void_p, c_int32, P(c_size_t)]),
    "cloth_train_workspace_size": (c_int32, [c_void_p, c_int32, P(c_size_t)]),
    "cloth_train_loss": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_float, c_float, c_void_p, c_void_p, c_void_p,
                                   c_size_t, c_void_p]),
    "cloth_train_loss_pcell": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_float, c_float, c_void_p, c_void_p,
                                         c_void_p, c_size_t, c_void_p]),
    "net_adam_step_masked": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_float,
                                       c_float, c_float, c_float, c_void_p]),
    "net_adam_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_float, c_float, c_float,
                                c_float, c_void_p]),
    "cloth_step_net": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_size_t, c_void_p]),
    "cloth_net_rollout_workspace_size": (c_int32, [c_void_p, c_int32, P(c_size_t)]),
    "cloth_pcell_workspace_size": (c_int32, [c_void_p, P(c_size_t)]),
    "cloth_pcell_accel": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "cloth_step_pcell": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_size_t, c_void_p]),
    "cloth_rollout_net": (c_int32, [c_void_p, c_void_p, P(NetRolloutOpts), c_void_p, c_size_t, c_void_p]),
    "cloth_modes": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "cloth_reset_modes": (c_int32, [c_void_p, c_void_p]),
    "cloth_info": (c_int32, [c_void_p, P(c_int32), P(c_int64)]),
    "cloth_destroy": (None, [c_void_p]),
    "cloth_strerror": (ctypes.c_char_p, [c_int32]),
    "cloth_last_cuda_error": (c_int32, []),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libcloth.so (building it first if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_needed and not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libcloth.so not found at {_build.LIB}; run the package build")
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class ClothError(RuntimeError):
    def __init__(self, fn: str, code: int):
        lib = load()
        msg = lib.cloth_strerror(code).decode()
        extra = f" (cudaError {lib.cloth_last_cuda_error()})" if code == -3 else ""
        super().__init__(f"{fn} failed: {ERRORS.get(code, code)}: {msg}{extra}")
        self.code = code


def check(fn: str, code: int) -> None:
    if code != CLOTH_OK:
        raise ClothError(fn, code)


def call(name: str, *args) -> None:
    check(name, getattr(load(), name)(*args))
