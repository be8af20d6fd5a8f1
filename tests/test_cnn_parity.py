"""GPU CNN cell (libcloth, FP32 CUDA cores) vs the FP64 oracle.

Tolerances (normwise = max |gpu - ref| / max |ref|):
  cell output a (FP32)          <= 1e-4
  gradients dLoss/dw, dLoss/dz  <= 1e-4
  network step positions        <= 1e-4 m max abs after 20 steps
Sizes span several 32 x 8 tiles with ragged tails, single nodes and the
128 x 128 inference batch (sampled).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import FP32, N_PARAMS, CellFunction, Net

pytestmark = pytest.mark.gpu

A_TOL = 1e-4
G_TOL = 1e-4


def normwise(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-30))


def blob(seed, h=0.02):
    """Kaiming weights with input scales that make the activations O(1):
    u / h and v / (1 m/s); outputs scaled by g."""
    return wl.kaiming_blob(seed, in_scale=(1 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.1)


def states(N, H, W, seed):
    rng = np.random.default_rng(seed)
    zs = []
    for _ in range(N):
        s = wl.cloth_spec(H, W)
        x, v = wl.sag_state(s, rng, amp=0.05, vamp=0.3)
        zs.append(oracle.net_input(s, x.astype(np.float64), v.astype(np.float64))[0])
    return np.stack(zs).astype(np.float32)


SHAPES = [(2, 13, 37), (1, 1, 1), (1, 2, 3), (3, 8, 32), (1, 33, 65)]


@pytest.mark.parametrize("N,H,W", SHAPES)
def test_forward_matches_oracle(N, H, W):
    w = blob(31)
    z = states(N, H, W, 32)
    net = Net(w, FP32)
    a, _ = net.forward(torch.from_numpy(z).cuda())
    ref = oracle.cnn_forward(w.astype(np.float64), z.astype(np.float64))
    assert normwise(a.cpu().numpy(), ref) <= A_TOL


def test_forward_random_inputs_and_nonlinear_regime():
    w = wl.kaiming_blob(33, in_scale=(2.0, 3.0, 1.0, 0.5, 1.5, 2.5), out_scale=(1.0, 0.5, 2.0), bias_sigma=0.5)
    z = np.random.default_rng(34).normal(size=(2, 6, 11, 45)).astype(np.float32)
    net = Net(w, FP32)
    a, _ = net.forward(torch.from_numpy(z).cuda())
    ref = oracle.cnn_forward(w.astype(np.float64), z.astype(np.float64))
    assert normwise(a.cpu().numpy(), ref) <= A_TOL


@pytest.mark.parametrize("N,H,W", [(2, 13, 37), (1, 1, 1), (1, 9, 33)])
def test_backward_matches_oracle(N, H, W):
    w = blob(35)
    z = states(N, H, W, 36)
    ga = np.random.default_rng(37).normal(size=(N, 3, H, W)).astype(np.float32)
    net = Net(w, FP32)
    zt = torch.from_numpy(z).cuda()
    _, saved = net.forward(zt)
    gw, gz = net.backward(zt, saved, torch.from_numpy(ga).cuda())
    rgw, rgz = oracle.cnn_backward(w.astype(np.float64), z.astype(np.float64), ga.astype(np.float64))
    assert normwise(gw.cpu().numpy(), rgw) <= G_TOL
    assert normwise(gz.cpu().numpy(), rgz) <= G_TOL
    # per parameter group, so a small group is not hidden by a large one
    bounds = [0, 1728, 10944, 11808, 11811, 12835, 12931, 13027]
    g = gw.cpu().numpy()
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        assert normwise(g[lo:hi], rgw[lo:hi]) <= 10 * G_TOL, (lo, hi)


def test_backward_accumulates_and_is_bitwise_reproducible():
    w = blob(38)
    z = states(2, 16, 40, 39)
    ga = torch.from_numpy(np.random.default_rng(40).normal(size=(2, 3, 16, 40)).astype(np.float32)).cuda()
    net = Net(w, FP32)
    zt = torch.from_numpy(z).cuda()
    outs = []
    for _ in range(2):
        _, saved = net.forward(zt)
        gw, _ = net.backward(zt, saved, ga)
        outs.append(gw)
    assert torch.equal(outs[0], outs[1])
    _, saved = net.forward(zt)
    gw2, _ = net.backward(zt, saved, ga, grad_w=outs[0].clone())
    assert torch.allclose(gw2, 2 * outs[0], rtol=1e-6, atol=0)


def test_autograd_function_matches_oracle():
    w = blob(41)
    z = states(1, 12, 20, 42)
    net = Net(w, FP32)
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    zt = torch.from_numpy(z).cuda().requires_grad_(True)
    a = CellFunction.apply(zt, wt, net)
    ga = torch.from_numpy(np.random.default_rng(43).normal(size=a.shape).astype(np.float32)).cuda()
    (a * ga).sum().backward()
    rgw, rgz = oracle.cnn_backward(w.astype(np.float64), z.astype(np.float64), ga.cpu().numpy().astype(np.float64))
    assert normwise(wt.grad[:N_PARAMS].cpu().numpy(), rgw) <= G_TOL
    assert torch.all(wt.grad[N_PARAMS:] == 0)
    assert normwise(zt.grad.cpu().numpy(), rgz) <= G_TOL


def _net_step_case(specs, pins, xs, vs, w, steps, sample=None):
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    net = Net(w, FP32)
    cb.step_net(net, steps)
    x, _ = cb.get_state()
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(x)]
    for b in (sample if sample is not None else range(len(specs))):
        xr, _ = oracle.net_step(w.astype(np.float64), specs[b], xs[b], vs[b], pins=pins[b], steps=steps)
        err = np.abs(got[b] - xr).max()
        assert err <= 1e-4, (b, err)
    assert cb.status() == 0


def test_net_step_uneven_batch_with_pins_pressure_sphere():
    rng = np.random.default_rng(44)
    specs, pins, xs, vs = [], [], [], []
    for (r, c) in [(5, 7), (16, 33), (16, 33), (9, 20)]:
        sph = {"center": (0.1, 0.1, -0.05), "radius": 0.06} if r == 9 else None
        s = wl.cloth_spec(r, c, p=rng.normal(0, 0.5), sphere=sph)
        x, v = wl.sag_state(s, rng, amp=0.02, vamp=0.1)
        specs.append(s); xs.append(x); vs.append(v)
        pins.append([0, c - 1])
    _net_step_case(specs, pins, xs, vs, blob(45), steps=20)


def test_net_step_inference_batch_sampled():
    """32 cloths of 128 x 128 (the CNN inference workload), 2 steps; two
    cloths compared with the oracle."""
    cfg = wl.cnn_batch()
    _net_step_case(cfg["specs"], cfg["pins"], cfg["x"], cfg["v"], blob(46), steps=2, sample=[0, 31])


def test_net_step_velocity_matches_oracle_on_every_edge():
    """One FP32 network step on cloths of uneven sizes in one launch (single
    nodes, single rows and columns, an exact 14 x 14 tile, ragged tiles):
    the velocity change dt (a + f_p / m) against the oracle's, normwise to
    the cell's 1e-4.  Every edge and corner term of the fused composite step
    is on this path."""
    rng = np.random.default_rng(47)
    shapes = [(1, 1), (1, 2), (3, 1), (2, 3), (14, 14), (15, 29), (30, 16), (5, 5)]
    specs, pins, xs, vs = [], [], [], []
    for (r, c) in shapes:
        sp = wl.cloth_spec(r, c, p=rng.normal(0, 0.5))
        x, v = wl.sag_state(sp, rng, amp=0.02, vamp=0.1)
        specs.append(sp); xs.append(x); vs.append(v); pins.append([])
    w = blob(48)
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    cb.step_net(Net(w, FP32), 1)
    _, v1 = cb.get_state()
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(v1)]
    for b, sp in enumerate(specs):
        _, vr = oracle.net_step(w.astype(np.float64), sp, xs[b], vs[b], pins=[], steps=1)
        dv_ref = vr - vs[b].astype(np.float64)
        dv = got[b] - vs[b].astype(np.float64)
        assert normwise(dv, dv_ref) <= 1e-4, (shapes[b], normwise(dv, dv_ref))
    assert cb.status() == 0


def test_net_step_maximum_size_cloth_sampled():
    """One 2048 x 2048 cloth through the FP32 network step: sampled nodes
    (corners, edges, random) equal the oracle's network step on the window of
    radius 3 (the receptive field of the two 3x3 trunk convolutions and the
    3x3 linear branch) around them."""
    n = 2048
    rng = np.random.default_rng(49)
    sp = wl.cloth_spec(n, n, p=0.3)
    x, v = wl.noisy_flat_state(sp, 1e-3, rng)
    v = (v + rng.normal(0, 0.05, v.shape)).astype(np.float32)
    w = blob(50)
    cb = ClothBatch([sp], [[0]])
    cb.set_state(pack([x]).cuda(), pack([v]).cuda())
    cb.step_net(Net(w, FP32), 1)
    xg = cb.get_state()[0].cpu().numpy().reshape(n, n, 3)
    x64, v64 = x.astype(np.float64), v.astype(np.float64)
    samples = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (1, 1), (0, 700), (1500, n - 1)] + \
              [tuple(int(t) for t in rng.integers(0, n, 2)) for _ in range(30)]
    for (r, c) in samples:
        r0, r1, c0, c1 = max(0, r - 3), min(n, r + 4), max(0, c - 3), min(n, c + 4)
        ws = dict(sp)
        ws["rows"], ws["cols"] = r1 - r0, c1 - c0
        sh = np.array([c0 * sp["h"], r0 * sp["h"], 0.0])
        wpins = [0] if (r0, c0) == (0, 0) else []
        xr, _ = oracle.net_step(w.astype(np.float64), ws, x64[r0:r1, c0:c1] - sh, v64[r0:r1, c0:c1],
                                pins=wpins, steps=1)
        assert np.abs(xg[r, c] - (xr[r - r0, c - c0] + sh)).max() <= 1e-5, (r, c)
    assert cb.status() == 0

