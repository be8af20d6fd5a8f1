"""net_forward_static: the cell forward for callers that cannot allocate
device memory (a plug-in whose host application owns the whole GPU memory
budget, or a real-time frame loop that must not stall on an allocation).

It is called through the C ABI and must agree with net_forward (which uses
a caller-allocated activation buffer) within the FP32 cell tolerance of
1e-4 normwise, on two calls in a row — the second call reuses the static
scratch the first one left behind.  Calls beyond the static capacity are
refused on the host.  This file is collected last on purpose.
"""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

from paper_2403_12820_gb300 import _lib
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.net import FP32, Net

pytestmark = pytest.mark.gpu

TOL = 1e-4
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MAX_NODES = int(re.search(r"#define\s+CLOTH_NET_STATIC_MAX_NODES\s+(\d+)",
                          open(os.path.join(ROOT, "include", "cloth.h")).read()).group(1))
# the capacity exactly filled, and one row over it
FULL = (1, 6, MAX_NODES // 128, 128)
OVER = (1, 6, MAX_NODES // 128 + 1, 128)
assert MAX_NODES % 128 == 0


def _call_static(d_blob, z):
    N, _, H, W = z.shape
    a = torch.empty(N, 3, H, W, dtype=torch.float32, device=z.device)
    rc = _lib.load().net_forward_static(ctypes.c_void_p(d_blob.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                        ctypes.c_void_p(a.data_ptr()), N, H, W,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, a


def _normwise(a, ref):
    return float((a - ref).abs().max() / ref.abs().max().clamp_min(1e-30))


def test_static_forward_matches_net_forward_twice():
    blob = wl.kaiming_blob(77, in_scale=(50.0,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.1)
    d_blob = torch.from_numpy(blob).cuda()
    net = Net(blob, FP32)
    rng = np.random.default_rng(78)
    for shape in [(2, 6, 40, 50), FULL]:
        z = torch.from_numpy(rng.normal(0.0, 0.02, size=shape).astype(np.float32)).cuda()
        ref, _ = net.forward(z)
        rc, a = _call_static(d_blob, z)
        torch.cuda.synchronize()
        assert rc == 0
        assert _normwise(a, ref) <= TOL


def test_static_forward_refuses_oversized_calls():
    d_blob = torch.zeros(13036, device="cuda")
    z = torch.zeros(*OVER, device="cuda")
    rc, _ = _call_static(d_blob, z)
    assert rc == -1
