"""Larger-step networks on the GPU (Sec. 5: larger-step integration with the
cell): with cloth_set_net_stride(k) every network step advances dt_net =
k dt, so it matches the oracle's network step at that time step; the Eq. 8
loss unrolls with dt_net against targets k plain steps apart, with the mean
acceleration of the k plain steps as its physics target (loss and gradient
within 1e-4 of the oracle)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import _lib
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import BF16, FP32, Net

pytestmark = pytest.mark.gpu


def batch(seed, shapes):
    rng = np.random.default_rng(seed)
    specs, pins, xs, vs = [], [], [], []
    for (r, c) in shapes:
        s = wl.cloth_spec(r, c, p=rng.normal(0, 0.5))
        x, v = wl.sag_state(s, rng, amp=0.01, vamp=0.05)
        specs.append(s); xs.append(x); vs.append(v)
        pins.append([0, c - 1])
    return specs, pins, xs, vs


def with_dt(s, k):
    return dict(s, dt=wl.f32(k * s["dt"]))


def blob(seed, h=wl.H_DEFAULT):
    return wl.kaiming_blob(seed, in_scale=(1.0 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3)


@pytest.mark.parametrize("kind", ["fp32", "bf16", "pcell"])
def test_network_step_with_stride(kind):
    k = 3
    specs, pins, xs, vs = batch(601, [(5, 7), (16, 33), (30, 61)])
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    cb.set_net_stride(k)
    if kind == "pcell":
        w = wl.pcell_blob(602)
        cb.step_pcell(w, 5)
        ref = lambda s, x, v, p: oracle.pcell_step(w.astype(np.float64), s, x, v, pins=p, steps=5)
    else:
        w = blob(603)
        net = Net(w, FP32 if kind == "fp32" else BF16)
        cb.step_net(net, 5)
        ref = lambda s, x, v, p: oracle.net_step(w.astype(np.float64), s, x, v, pins=p, steps=5)
    x, _ = cb.get_state()
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(x)]
    for b, s in enumerate(specs):
        xr, _ = ref(with_dt(s, k), xs[b].astype(np.float64), vs[b].astype(np.float64), pins[b])
        assert np.abs(got[b] - xr).max() <= 1e-4, (b, np.abs(got[b] - xr).max())
    assert cb.status() == 0
    cb.close()


@pytest.mark.parametrize("cell", ["pcell", "cnn"])
def test_training_loss_with_stride(cell):
    k, S, alpha, g = 3, 3, 0.5, 9.81
    cfg = wl.plain_batch(seed=605, count=2, side_lo=10, side_hi=10)
    rng = np.random.default_rng(606)
    xs, vs, tgs, ats = [], [], [], []
    for b in range(2):
        s = cfg["specs"][b]
        x0, v0 = wl.sag_state(s, rng, amp=0.02, vamp=0.05)
        x0 = x0.astype(np.float32).astype(np.float64)
        v0 = v0.astype(np.float32).astype(np.float64)
        tg, xt, vt = [], x0, v0
        for _ in range(S):
            xt, vt = oracle.step(s, xt, vt, pins=cfg["pins"][b], steps=k)
            tg.append(xt.astype(np.float32).astype(np.float64))
        xs.append(x0); vs.append(v0); tgs.append(np.array(tg))
        ats.append(oracle.mean_accel(s, x0, v0, cfg["pins"][b], k=k))
    if cell == "pcell":
        w = wl.pcell_blob(607).astype(np.float64)
        w[12:36] *= np.random.default_rng(608).uniform(0.5, 2.0, 24)
        w = w.astype(np.float32)
        n_par = 39
    else:
        w = blob(609, cfg["specs"][0]["h"]).astype(np.float32)
        n_par = 13027
    rl, rg = 0.0, 0.0
    for b, s in enumerate(cfg["specs"]):
        l, gw = oracle.unroll_loss(w.astype(np.float64), with_dt(s, k), cfg["pins"][b], xs[b], vs[b], tgs[b], ats[b],
                                   alpha, g, s["h"], cell=cell)
        rl += l / 2; rg = rg + gw / 2
    cb = ClothBatch(cfg["specs"], cfg["pins"])
    cb.set_state(pack([x.astype(np.float32) for x in xs]).cuda(), pack([v.astype(np.float32) for v in vs]).cuda())
    cb.set_net_stride(k)
    tg = torch.from_numpy(np.stack([np.concatenate([tgs[b][t].reshape(-1, 3) for b in range(2)])
                                    for t in range(S)]).astype(np.float32)).cuda()
    if cell == "pcell":
        loss, grad = cb.train_loss_pcell(w, S, tg, alpha=alpha, g_norm=g)
    else:
        net = Net(w, FP32)
        loss, grad = cb.train_loss(net, S, tg, alpha=alpha, g_norm=g)
    assert abs(loss.item() - rl) <= 1e-4 * abs(rl), (loss.item(), rl)
    gg = grad.cpu().numpy()[:n_par]
    assert np.abs(gg - rg[:n_par]).max() <= 1e-4 * np.abs(rg[:n_par]).max()
    x, _ = cb.get_state()
    assert torch.equal(x, pack([x.astype(np.float32) for x in xs]).cuda())
    cb.close()


def test_stride_limits_and_reset():
    specs, pins, xs, vs = batch(611, [(16, 33), (9, 20)])
    w = blob(612)
    net = Net(w, BF16)
    cb = ClothBatch(specs, pins)
    x0, v0 = pack(xs).cuda(), pack(vs).cuda()
    cb.set_state(x0, v0)
    cb.step_net(net, 4)
    ref = cb.get_state()
    for bad in (0, -1, 1001):
        with pytest.raises(_lib.ClothError):
            cb.set_net_stride(bad)
    cb.set_net_stride(4)
    cb.rollout_net(net, 10)
    cb.set_net_stride(1)
    cb.set_state(x0, v0)
    cb.step_net(net, 4)
    got = cb.get_state()
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
    cb.close(); net.close()


def test_trainer_with_stride_runs():
    from paper_2403_12820_gb300.train import Dataset, Trainer

    data = Dataset(count=4, n=12, steps=16, seed=1004)
    tr = Trainer(data, batch=2, unroll=3, cell="pcell", stride=4)
    losses = [tr.step() for _ in range(2)]
    assert all(np.isfinite(losses))
    with pytest.raises(ValueError):
        Trainer(data, batch=2, unroll=5, cell="pcell", stride=4)


@pytest.mark.parametrize("chunk", [0, 4])
def test_checked_rollout_at_stride(chunk):
    """Residual check at stride k: bound 0 switches every cloth at the first
    check, after which each network step is k plain steps (the plain rollout
    bit for bit); an infinite bound keeps the network (the unchecked rollout
    bit for bit)."""
    k = 3
    specs, pins, xs, vs = batch(613, [(16, 33), (9, 20), (40, 41)])
    w = blob(614)
    net = Net(w, BF16)
    x0, v0 = pack(xs).cuda(), pack(vs).cuda()

    def run(fn, stride):
        cb = ClothBatch(specs, pins)
        cb.set_state(x0, v0)
        if stride != 1:
            cb.set_net_stride(stride)
        fn(cb)
        out = cb.get_state()
        modes = cb.modes()[0].cpu().numpy()
        assert cb.status() == 0
        cb.close()
        return out, modes

    (xa, va), ma = run(lambda cb: cb.rollout_net(net, 8, check_every=2, residual_bound=0.0, graph_chunk=chunk), k)
    (xb, vb), _ = run(lambda cb: cb.rollout(8 * k), 1)
    assert ma.tolist() == [1, 1, 1]
    assert torch.equal(xa, xb) and torch.equal(va, vb)
    (xa, va), ma = run(lambda cb: cb.rollout_net(net, 8, check_every=2, residual_bound=float("inf"),
                                                 graph_chunk=chunk), k)
    (xb, vb), _ = run(lambda cb: cb.step_net(net, 8), k)
    assert ma.tolist() == [0, 0, 0]
    assert torch.equal(xa, xb) and torch.equal(va, vb)
    net.close()
