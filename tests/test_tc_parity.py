"""Tensor-core (tcgen05, BF16 operands, FP32 accumulation) CNN cell and
network step vs the FP64 oracle.

Tolerances: cell output a <= 2e-2 normwise (BF16); network-step positions
<= 1e-4 m after 20 steps.  Sizes cover one exact 14 x 26 tile, several
tiles with ragged edges, single nodes, and the 128 x 128 inference batch.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import BF16, FP32, Net

pytestmark = pytest.mark.gpu

A_TOL = 2e-2


def normwise(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-30))


def blob(seed, h=0.02):
    return wl.kaiming_blob(seed, in_scale=(1 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.1)


def states(N, H, W, seed, amp=0.05, vamp=0.3):
    rng = np.random.default_rng(seed)
    zs = []
    for _ in range(N):
        s = wl.cloth_spec(H, W)
        x, v = wl.sag_state(s, rng, amp=amp, vamp=vamp)
        zs.append(oracle.net_input(s, x.astype(np.float64), v.astype(np.float64))[0])
    return np.stack(zs).astype(np.float32)


@pytest.mark.parametrize("N,H,W", [(1, 14, 26), (1, 12, 28), (2, 13, 37), (1, 1, 1), (1, 2, 3), (1, 30, 61), (3, 25, 57)])
def test_bf16_cell_matches_oracle(N, H, W):
    w = blob(51)
    z = states(N, H, W, 52)
    net = Net(w, BF16)
    a, _ = net.forward(torch.from_numpy(z).cuda())
    torch.cuda.synchronize()
    ref = oracle.cnn_forward(w.astype(np.float64), z.astype(np.float64))
    assert normwise(a.cpu().numpy(), ref) <= A_TOL


def test_bf16_cell_random_weights_and_inputs():
    w = wl.kaiming_blob(53, in_scale=(2.0, 3.0, 1.0, 0.5, 1.5, 2.5), out_scale=(1.0, 0.5, 2.0), bias_sigma=0.5)
    z = np.random.default_rng(54).normal(size=(2, 6, 11, 45)).astype(np.float32)
    net = Net(w, BF16)
    a, _ = net.forward(torch.from_numpy(z).cuda())
    ref = oracle.cnn_forward(w.astype(np.float64), z.astype(np.float64))
    assert normwise(a.cpu().numpy(), ref) <= A_TOL


def test_bf16_cell_inference_batch_sampled():
    """The 32 x 128 x 128 batch through the tensor-core cell; two images vs
    the oracle, all images vs the FP32 CUDA-core cell."""
    w = blob(55)
    z = states(32, 128, 128, 56)
    zt = torch.from_numpy(z).cuda()
    a16, _ = Net(w, BF16).forward(zt)
    a32, _ = Net(w, FP32).forward(zt)
    torch.cuda.synchronize()
    for n in (0, 31):
        ref = oracle.cnn_forward(w.astype(np.float64), z[n:n + 1].astype(np.float64))
        assert normwise(a16[n:n + 1].cpu().numpy(), ref) <= A_TOL
    assert float((a16 - a32).abs().max() / a32.abs().max()) <= A_TOL


def test_bf16_net_step_matches_oracle():
    rng = np.random.default_rng(57)
    specs, pins, xs, vs = [], [], [], []
    for (r, c) in [(5, 7), (16, 33), (30, 61), (12, 28)]:
        sph = {"center": (0.1, 0.1, -0.05), "radius": 0.06} if r == 16 else None
        s = wl.cloth_spec(r, c, p=rng.normal(0, 0.5), sphere=sph)
        x, v = wl.sag_state(s, rng, amp=0.02, vamp=0.1)
        specs.append(s); xs.append(x); vs.append(v)
        pins.append([0, c - 1])
    w = blob(58)
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    net = Net(w, BF16)
    cb.step_net(net, 20)
    x, _ = cb.get_state()
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(x)]
    for b in range(len(specs)):
        xr, _ = oracle.net_step(w.astype(np.float64), specs[b], xs[b], vs[b], pins=pins[b], steps=20)
        assert np.abs(got[b] - xr).max() <= 1e-4, b
    assert cb.status() == 0


def test_bf16_net_step_is_deterministic():
    cfg = wl.cnn_batch(count=4)
    w = blob(59)
    outs = []
    for _ in range(2):
        cb = ClothBatch(cfg["specs"], cfg["pins"])
        cb.set_state(pack(cfg["x"]).cuda(), pack(cfg["v"]).cuda())
        cb.step_net(Net(w, BF16), 5)
        outs.append(cb.get_state()[0])
    assert torch.equal(outs[0], outs[1])


def test_bf16_maximum_size_cloth_sampled():
    """One 2048 x 2048 cloth through the tensor-core network step: sampled
    nodes equal the oracle's network step on the window of radius 3 (the
    receptive field of the two 3x3 trunk convolutions and the 3x3 linear
    branch) around them."""
    n = 2048
    rng = np.random.default_rng(94)
    s = wl.cloth_spec(n, n, p=0.3)
    x, v = wl.noisy_flat_state(s, 1e-3, rng)
    v = (v + rng.normal(0, 0.05, v.shape)).astype(np.float32)
    w = blob(95)
    cb = ClothBatch([s], [[0]])
    cb.set_state(pack([x]).cuda(), pack([v]).cuda())
    cb.step_net(Net(w, BF16), 1)
    xg = cb.get_state()[0].cpu().numpy().reshape(n, n, 3)
    x64, v64 = x.astype(np.float64), v.astype(np.float64)
    samples = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (2, 1000), (n // 2, n // 2)] + \
              [tuple(int(t) for t in rng.integers(0, n, 2)) for _ in range(30)]
    for (r, c) in samples:
        r0, r1, c0, c1 = max(0, r - 3), min(n, r + 4), max(0, c - 3), min(n, c + 4)
        ws = dict(s)
        ws["rows"], ws["cols"] = r1 - r0, c1 - c0
        sh = np.array([c0 * s["h"], r0 * s["h"], 0.0])
        wpins = [0] if (r0, c0) == (0, 0) else []
        xr, _ = oracle.net_step(w.astype(np.float64), ws, x64[r0:r1, c0:c1] - sh, v64[r0:r1, c0:c1],
                                pins=wpins, steps=1)
        assert np.abs(xg[r, c] - (xr[r - r0, c - c0] + sh)).max() <= 1e-4, (r, c)
    assert cb.status() == 0
