"""Network rollout judged by the plain step (Fig. 2 couples the network with
the physics-based simulator): per-cloth residual checks and the switch to
the plain step, vs the FP64 oracle's plain and network steps.

A bound of 0 switches every cloth at the first check, so the rollout must be
the plain rollout bit for bit; an infinite bound switches none, so it must
be the network rollout bit for bit.  Between the two, the cloths whose
oracle residual lies above the bound switch and the others do not, and each
then follows its own oracle step (positions within 1e-4 m).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300._lib import ClothError
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import BF16, FP32, Net

pytestmark = pytest.mark.gpu


def blob(seed):
    h = wl.H_DEFAULT
    return wl.kaiming_blob(seed, in_scale=(1 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.1)


def sphere_batch(seed=71, sides=(20, 33, 47, 60, 25, 40), sigmas=(1e-5, 3e-5, 1e-4, 3e-4, 1e-3, 3e-3)):
    """Square cloths over a sphere (the large-cloth sphere workload, scaled
    down), each with its own noise level so that residuals spread."""
    rng = np.random.default_rng(seed)
    specs, pins, xs, vs = [], [], [], []
    for n, sg in zip(sides, sigmas):
        w = (n - 1) * wl.H_DEFAULT
        R = 0.3 * w
        s = wl.cloth_spec(n, n, p=rng.normal(0, 0.5), sphere={"center": (w / 2, w / 2, -R - 0.05 * w), "radius": R})
        x, v = wl.noisy_flat_state(s, sg, rng)
        specs.append(s); pins.append([0, n - 1]); xs.append(x); vs.append(v)
    return specs, pins, xs, vs


def make(specs, pins, xs, vs):
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    return cb


@pytest.mark.parametrize("precision", [BF16, FP32])
@pytest.mark.parametrize("chunk", [0, 8])
def test_bound_zero_is_the_plain_rollout(chunk, precision):
    sb = sphere_batch()
    net = Net(blob(72), precision)
    a = make(*sb)
    a.rollout_net(net, 30, check_every=1, residual_bound=0.0, graph_chunk=chunk)
    b = make(*sb)
    b.step(30)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert torch.equal(xa, xb) and torch.equal(va, vb)
    mode, resid = a.modes()
    assert mode.cpu().tolist() == [1] * len(sb[0])
    assert bool((resid > 0).all())
    assert a.status() == 0


@pytest.mark.parametrize("precision", [BF16, FP32])
@pytest.mark.parametrize("check_every,chunk", [(3, 0), (3, 6), (1, 4), (0, 0)])
def test_infinite_bound_is_the_network_rollout(check_every, chunk, precision):
    sb = sphere_batch()
    net = Net(blob(73), precision)
    a = make(*sb)
    a.rollout_net(net, 20, check_every=check_every, residual_bound=float("inf"), graph_chunk=chunk)
    b = make(*sb)
    b.step_net(net, 20)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert torch.equal(xa, xb) and torch.equal(va, vb)
    mode, resid = a.modes()
    assert mode.cpu().tolist() == [0] * len(sb[0])
    if check_every:
        assert bool(torch.isfinite(resid).all()) and bool((resid > 0).all())


@pytest.mark.parametrize("precision", [BF16, FP32])
def test_switch_follows_the_oracle(precision):
    specs, pins, xs, vs = sphere_batch()
    w = blob(74)
    w64 = w.astype(np.float64)
    B = len(specs)
    # oracle residual of one check from the initial state
    xp1, vp1, xn1, vn1, r, tol = [], [], [], [], [], []
    for b in range(B):
        xp, vp = oracle.step(specs[b], xs[b], vs[b], pins=pins[b])
        xn, vn = oracle.net_step(w64, specs[b], xs[b], vs[b], pins=pins[b])
        xp1.append(xp); vp1.append(vp); xn1.append(xn); vn1.append(vn)
        r.append(float(np.sqrt(((xn - xp) ** 2).sum(axis=-1)).max()))
        # the cell's 2e-2 normwise tolerance carried through one Euler step
        tol.append(2e-2 * float(specs[b]["dt"]) ** 2 * np.abs(oracle.net_accel(w64, specs[b], xs[b], vs[b])).max())
    r = np.asarray(r)
    rs = np.sort(r)
    gaps = rs[2:-1] / rs[1:-2]
    i = int(np.argmax(gaps)) + 1
    assert gaps.max() > 1.2, rs
    bound = float(np.sqrt(rs[i] * rs[i + 1]))
    expect = (r > bound).astype(int)
    assert 0 < expect.sum() < B

    cb = make(specs, pins, xs, vs)
    net = Net(w, precision)
    cb.rollout_net(net, 1, check_every=1, residual_bound=bound)
    mode, resid = cb.modes()
    assert mode.cpu().numpy().tolist() == expect.tolist()
    assert (np.abs(resid.cpu().numpy() - r) <= np.asarray(tol) + 1e-6 * r + 1e-9).all(), (resid, r, tol)
    # the switched cloths run plain, the others keep the network step
    cb.rollout_net(net, 10, check_every=0)
    x, _ = cb.get_state()
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(x)]
    for b in range(B):
        if expect[b]:
            xr, _ = oracle.step(specs[b], xp1[b], vp1[b], pins=pins[b], steps=10)
        else:
            xr, _ = oracle.net_step(w64, specs[b], xn1[b], vn1[b], pins=pins[b], steps=10)
        assert np.abs(got[b] - xr).max() <= 1e-4, b
    # switching back
    cb.reset_modes()
    mode, resid = cb.modes()
    assert int(mode.sum()) == 0 and float(resid.abs().sum()) == 0.0
    assert cb.status() == 0


@pytest.mark.parametrize("precision", [BF16, FP32])
def test_a_negative_bound_is_rejected(precision):
    sb = sphere_batch(sides=(16, 16), sigmas=(1e-4, 1e-4))
    cb = make(*sb)
    with pytest.raises(ClothError, match="EINVAL"):
        cb.rollout_net(Net(blob(75), precision), 2, check_every=1, residual_bound=-1.0)
