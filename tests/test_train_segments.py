"""Segment checkpointing of the Eq. 8 unroll: keeping only every k-th state
and recomputing the others in the backward sweep gives bitwise the same loss
and gradient as keeping every state, for both cells, with less workspace."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import _lib
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import FP32, Net

pytestmark = pytest.mark.gpu


def windows(S, B=2, n=10, seed=801):
    cfg = wl.plain_batch(seed=seed, count=B, side_lo=n, side_hi=n)
    rng = np.random.default_rng(seed + 1)
    xs, vs, tgs = [], [], []
    for b in range(B):
        s = cfg["specs"][b]
        x0, v0 = wl.sag_state(s, rng, amp=0.02, vamp=0.05)
        tg, xt, vt = [], x0.astype(np.float64), v0.astype(np.float64)
        for _ in range(S):
            xt, vt = oracle.step(s, xt, vt, pins=cfg["pins"][b], steps=1)
            tg.append(xt)
        xs.append(x0); vs.append(v0); tgs.append(np.array(tg))
    tg = torch.from_numpy(np.stack([np.concatenate([tgs[b][t].reshape(-1, 3) for b in range(B)])
                                    for t in range(S)]).astype(np.float32)).cuda()
    return cfg, pack(xs).cuda(), pack(vs).cuda(), tg


def ws_bytes(cb, S):
    n = ctypes.c_size_t()
    _lib.call("cloth_train_workspace_size", cb.handle, int(S), ctypes.byref(n))
    return n.value


@pytest.mark.parametrize("cell", ["pcell", "cnn"])
def test_segments_give_the_same_bits(cell):
    S = 11
    cfg, x0, v0, tg = windows(S)
    h = cfg["specs"][0]["h"]
    w = (wl.pcell_blob(803) if cell == "pcell" else
         wl.kaiming_blob(804, in_scale=(1.0 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3)).astype(np.float32)
    net = Net(w, FP32) if cell == "cnn" else None
    outs, sizes = [], []
    for k in (0, 1, 3, 4, 11, 20):
        cb = ClothBatch(cfg["specs"], cfg["pins"])
        cb.set_state(x0, v0)
        cb.set_train_segment(k)
        sizes.append(ws_bytes(cb, S))
        if cell == "pcell":
            loss, g = cb.train_loss_pcell(w, S, tg)
        else:
            loss, g = cb.train_loss(net, S, tg)
        outs.append((loss.clone(), g.clone()))
        x, v = cb.get_state()
        assert torch.equal(x, x0) and torch.equal(v, v0)
        cb.close()
    for k, (l, g) in zip((1, 3, 4, 11, 20), outs[1:]):
        assert torch.equal(l, outs[0][0]) and torch.equal(g, outs[0][1]), k
    assert sizes[2] < sizes[0] and sizes[3] < sizes[0]   # k = 3, 4: 6 and 5 states instead of 12
    if net is not None:
        net.close()


def test_rejects_negative_segments():
    cfg, x0, v0, tg = windows(2)
    cb = ClothBatch(cfg["specs"], cfg["pins"])
    with pytest.raises(_lib.ClothError):
        cb.set_train_segment(-1)
    cb.close()
