"""Training path on the GPU vs the FP64 oracle (Eq. 8, Table 1).

The loss and its gradient through an S-step unroll (network, pressure,
pins, Euler) must match the oracle's hand-written adjoint: loss within
1e-4 relative, gradient within 1e-4 normwise.  Window targets come from the
oracle's own plain step.  Adam matches the closed-form update.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import FP32, N_PARAMS, Net, adam_step

pytestmark = pytest.mark.gpu


def windows(B=3, n=10, S=4, seed=61):
    cfg = wl.plain_batch(seed=seed, count=B, side_lo=n, side_hi=n)
    rng = np.random.default_rng(seed + 1)
    xs, vs, tgs, ats = [], [], [], []
    for b in range(B):
        s = cfg["specs"][b]
        x0, v0 = wl.sag_state(s, rng, amp=0.02, vamp=0.05)
        x0 = x0.astype(np.float64); v0 = v0.astype(np.float64)
        tg, xt, vt = [], x0, v0
        for _ in range(S):
            xt, vt = oracle.step(s, xt, vt, pins=cfg["pins"][b], steps=1)
            tg.append(xt)
        xs.append(x0.astype(np.float32)); vs.append(v0.astype(np.float32)); tgs.append(np.array(tg))
        f = oracle.total_force(s, x0, v0) - oracle.pressure_force(s, x0)
        ats.append(f / s["m"])
    return cfg, xs, vs, tgs, ats


def test_train_loss_and_gradient_match_oracle():
    S, alpha, g = 4, 0.5, 9.81
    cfg, xs, vs, tgs, ats = windows(S=S)
    w = wl.kaiming_blob(62, in_scale=(50.0,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.1)
    # oracle: mean over windows of the per-window loss and gradient (targets
    # rounded to float32 as the GPU receives them)
    rl, rg = 0.0, np.zeros(N_PARAMS)
    for b, s in enumerate(cfg["specs"]):
        tg32 = tgs[b].astype(np.float32).astype(np.float64)
        l, gw = oracle.unroll_loss(w.astype(np.float64), s, cfg["pins"][b], xs[b].astype(np.float64),
                                   vs[b].astype(np.float64), tg32, ats[b], alpha, g, s["h"])
        rl += l / len(cfg["specs"]); rg += gw / len(cfg["specs"])
    cb = ClothBatch(cfg["specs"], cfg["pins"])
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    net = Net(w, FP32)
    targets = torch.from_numpy(np.stack([np.concatenate([tgs[b][t].reshape(-1, 3) for b in range(len(xs))])
                                         for t in range(S)]).astype(np.float32)).cuda()
    loss, grad = cb.train_loss(net, S, targets, alpha=alpha, g_norm=g)
    torch.cuda.synchronize()
    assert abs(loss.item() - rl) <= 1e-4 * abs(rl), (loss.item(), rl)
    gg = grad.cpu().numpy()
    assert np.abs(gg - rg).max() <= 1e-4 * np.abs(rg).max()
    # the context's state is left untouched
    x, _ = cb.get_state()
    assert torch.equal(x, pack(xs).cuda())


def test_train_loss_is_bitwise_reproducible():
    cfg, xs, vs, tgs, _ = windows(B=2, n=12, S=3, seed=63)
    w = wl.kaiming_blob(64, in_scale=(50.0,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3)
    targets = torch.from_numpy(np.stack([np.concatenate([tgs[b][t].reshape(-1, 3) for b in range(2)])
                                         for t in range(3)]).astype(np.float32)).cuda()
    outs = []
    for _ in range(2):
        cb = ClothBatch(cfg["specs"], cfg["pins"])
        cb.set_state(pack(xs).cuda(), pack(vs).cuda())
        outs.append(cb.train_loss(Net(w, FP32), 3, targets))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_adam_matches_oracle():
    rng = np.random.default_rng(65)
    th, g = rng.normal(size=1000), rng.normal(size=1000)
    m, v = rng.normal(size=1000) * 0.1, np.abs(rng.normal(size=1000)) * 0.01
    # hyper-parameters as the kernel receives them: float32 values
    f = lambda a: float(np.float32(a))
    ref = oracle.adam_step(th, g, m, v, t=7, lr=f(1e-3), beta1=f(0.9), beta2=f(0.999), eps=f(1e-8))
    t_ = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (th, g, m, v)]
    adam_step(t_[0], t_[1], t_[2], t_[3], t=7, lr=1e-3)
    np.testing.assert_allclose(t_[0].cpu().numpy(), ref[0], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(t_[2].cpu().numpy(), ref[1], rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(t_[3].cpu().numpy(), ref[2], rtol=1e-5, atol=1e-9)


def test_training_reduces_the_loss():
    """Adam (Table 1's starting rate 1e-2) on one fixed batch of windows of
    recorded plain-step trajectories: the Eq. 8 loss must fall."""
    from paper_2403_12820_gb300.train import Dataset, Trainer
    data = Dataset(count=8, n=16, steps=40, seed=66)
    tr = Trainer(data, batch=8, unroll=4, lr=1e-2, seed=67)
    specs, pins, x0, v0, tg = tr.sample()
    cb = ClothBatch(specs, pins)
    losses = []
    for it in range(120):
        cb.set_state(x0, v0)
        tr.net.set_weights(tr.w)
        loss, g = cb.train_loss(tr.net, 4, tg)
        adam_step(tr.w, g, tr.m, tr.v, it + 1, lr=1e-2, n=N_PARAMS)
        losses.append(loss.item())
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:5]), (losses[:5], losses[-5:])


def test_state_pool_windows_are_labelled_by_the_plain_step():
    """The trainer's network-stepped state pool: after its warm-up the pool
    supplies part of each batch; a pool window's targets are the plain
    step's positions from the window's start (checked against the oracle),
    the losses stay finite, and slots restart once they reach their age."""
    from paper_2403_12820_gb300.train import Dataset, Trainer
    data = Dataset(count=6, n=12, steps=12, seed=1004)
    tr = Trainer(data, batch=4, unroll=3, seed=9, pool=4, pool_frac=0.5, pool_steps=4, pool_age=8, pool_warm=2)
    losses = [tr.step() for _ in range(8)]
    assert all(np.isfinite(losses))
    assert tr.pool is not None and tr.pool.restarts > tr.pool.count
    specs, pins, x0, v0, tg = tr.pool.windows(2, 3, 1)
    nn = 12 * 12
    for b in range(2):
        xb = x0[b * nn:(b + 1) * nn].cpu().numpy().astype(np.float64).reshape(12, 12, 3)
        vb = v0[b * nn:(b + 1) * nn].cpu().numpy().astype(np.float64).reshape(12, 12, 3)
        xr, vr = xb, vb
        for s in range(3):
            xr, vr = oracle.step(specs[b], xr, vr, pins=pins[b], steps=1)
            got = tg[s, b * nn:(b + 1) * nn].cpu().numpy().astype(np.float64).reshape(12, 12, 3)
            assert np.abs(got - xr).max() <= 1e-6, (b, s)
    tr.pool.close()
