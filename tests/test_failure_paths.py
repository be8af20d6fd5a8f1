"""Failure paths made without faulting the GPU: a bounded wait that runs out
(an mbarrier nothing completes) reports CLOTH_STATUS_TIMEOUT and the context
stays usable; a non-finite state reports CLOTH_STATUS_NONFINITE; corrupted
network weights make the residual check switch every cloth to the plain
step; bad arguments are refused before anything runs."""
import numpy as np
import pytest
import torch

from paper_2403_12820_gb300 import _lib
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import BF16, FP32, Net

pytestmark = pytest.mark.gpu


def batch():
    rng = np.random.default_rng(901)
    specs, pins, xs, vs = [], [], [], []
    for (r, c) in [(16, 33), (40, 41)]:
        s = wl.cloth_spec(r, c, p=0.2)
        x, v = wl.sag_state(s, rng, amp=0.01, vamp=0.05)
        specs.append(s); xs.append(x); vs.append(v); pins.append([0, c - 1])
    return specs, pins, pack(xs).cuda(), pack(vs).cuda()


def test_bounded_wait_reports_timeout_and_the_context_stays_usable():
    specs, pins, x0, v0 = batch()
    cb = ClothBatch(specs, pins)
    cb.set_state(x0, v0)
    assert cb.status() == 0
    cb.selftest_wait_timeout(200)
    assert cb.status(clear=True) == _lib.STATUS_TIMEOUT
    assert cb.status() == 0
    cb.step(5)
    ref = ClothBatch(specs, pins)
    ref.set_state(x0, v0)
    ref.step(5)
    assert torch.equal(cb.get_state()[0], ref.get_state()[0]) and cb.status() == 0
    with pytest.raises(_lib.ClothError):
        cb.selftest_wait_timeout(0)
    cb.close(); ref.close()


def test_nonfinite_state_is_reported():
    specs, pins, x0, v0 = batch()
    x = x0.clone()
    x[7, 2] = float("inf")
    cb = ClothBatch(specs, pins)
    cb.set_state(x, v0)
    cb.step(1)
    assert cb.status(clear=True) & _lib.STATUS_NONFINITE
    cb.close()


def test_corrupted_weights_switch_every_cloth_to_the_plain_step():
    specs, pins, x0, v0 = batch()
    h = specs[0]["h"]
    w = wl.kaiming_blob(902, in_scale=(1.0 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3).astype(np.float32)
    w[:13027] *= 1e4                          # a broken network: huge accelerations
    net = Net(w, BF16)
    cb = ClothBatch(specs, pins)
    cb.set_state(x0, v0)
    cb.rollout_net(net, 20, check_every=5, residual_bound=1e-3)
    mode, resid = cb.modes()
    assert mode.cpu().tolist() == [1, 1]
    assert float(resid.min()) > 1e-3
    # from the switch on, the cloths follow the plain step
    ref = ClothBatch(specs, pins)
    ref.set_state(x0, v0)
    ref.rollout(20)
    assert torch.equal(cb.get_state()[0], ref.get_state()[0])
    cb.close(); ref.close(); net.close()


@pytest.mark.parametrize("precision", [BF16, FP32])
def test_nan_weight_switches_every_cloth_to_the_plain_step(precision):
    """One NaN weight turns every network result NaN.  net_create refuses a
    non-finite blob, so the NaN comes the way a diverged training run would
    leave it: device weights given to net_set_weights (the blob is made on the
    host).  The residual check must see a non-finite residual, not drop it,
    switch every cloth at the first check, and leave the plain rollout bit
    for bit."""
    specs, pins, x0, v0 = batch()
    h = specs[0]["h"]
    w = wl.kaiming_blob(903, in_scale=(1.0 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3).astype(np.float32)
    net = Net(w, precision)
    w[1728 + 5] = np.nan                      # one entry of W2
    net.set_weights(torch.from_numpy(w).cuda())
    cb = ClothBatch(specs, pins)
    cb.set_state(x0, v0)
    cb.rollout_net(net, 20, check_every=5, residual_bound=1e-3)
    mode, resid = cb.modes()
    assert mode.cpu().tolist() == [1, 1]
    r = resid.cpu().numpy()
    assert np.all(~np.isfinite(r) | (r > 1e-3)), r
    ref = ClothBatch(specs, pins)
    ref.set_state(x0, v0)
    ref.rollout(20)
    x, v = cb.get_state()
    xr, vr = ref.get_state()
    assert torch.equal(x, xr) and torch.equal(v, vr)
    assert bool(torch.isfinite(x).all())
    cb.close(); ref.close(); net.close()


@pytest.mark.parametrize("cell", ["pcell", "cnn"])
def test_trainer_checkpoint_resumes_bit_for_bit(tmp_path, cell):
    from paper_2403_12820_gb300.train import Dataset, Trainer

    data = Dataset(count=6, n=12, steps=12, seed=1004)
    a = Trainer(data, batch=3, unroll=3, cell=cell, seed=11)
    a.step(); a.step()
    path = str(tmp_path / "ck.npz")
    a.save(path)
    la = [a.step(), a.step()]
    b = Trainer(data, batch=3, unroll=3, cell=cell, seed=99)   # another sampler seed: load restores it
    b.load(path)
    lb = [b.step(), b.step()]
    assert la == lb
    assert torch.equal(a.w, b.w) and torch.equal(a.m, b.m) and torch.equal(a.v, b.v) and a.t == b.t
    other = Trainer(data, batch=3, unroll=3, cell="pcell" if cell == "cnn" else "cnn")
    with pytest.raises(ValueError):
        other.load(path)
