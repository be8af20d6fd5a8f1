"""Eq. 8 training with the literal cell (Eq. 6-7, Fig. 1) on the GPU vs the
FP64 oracle: the loss within 1e-4 relative and the parameter gradient
within 1e-4 normwise of the oracle's hand-written adjoint through an S-step
unroll (cell, pressure, pins, Euler); bitwise reproducibility; a few Adam
steps reduce the loss."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import adam_step

pytestmark = pytest.mark.gpu


def windows(B=3, n=10, S=4, seed=101):
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


def targets_of(tgs, S, B):
    return torch.from_numpy(np.stack([np.concatenate([tgs[b][t].reshape(-1, 3) for b in range(B)])
                                      for t in range(S)]).astype(np.float32)).cuda()


def weights(seed):
    rng = np.random.default_rng(seed)
    w = wl.pcell_blob(seed).astype(np.float64)
    w[12:36] *= rng.uniform(0.5, 2.0, 24)
    return w.astype(np.float32)


def test_loss_and_gradient_match_oracle():
    S, alpha, g = 4, 0.5, 9.81
    cfg, xs, vs, tgs, ats = windows(S=S)
    B = len(xs)
    w = weights(103)
    rl, rg = 0.0, np.zeros(40)
    for b, s in enumerate(cfg["specs"]):
        tg32 = tgs[b].astype(np.float32).astype(np.float64)
        l, gw = oracle.unroll_loss(w.astype(np.float64), s, cfg["pins"][b], xs[b].astype(np.float64),
                                   vs[b].astype(np.float64), tg32, ats[b], alpha, g, s["h"], cell="pcell")
        rl += l / B; rg += gw / B
    cb = ClothBatch(cfg["specs"], cfg["pins"])
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    loss, grad = cb.train_loss_pcell(w, S, targets_of(tgs, S, B), alpha=alpha, g_norm=g)
    torch.cuda.synchronize()
    assert abs(loss.item() - rl) <= 1e-4 * abs(rl), (loss.item(), rl)
    gg = grad.cpu().numpy()
    assert gg[39] == 0.0
    assert np.abs(gg[:39] - rg[:39]).max() <= 1e-4 * np.abs(rg[:39]).max(), np.abs(gg[:39] - rg[:39]).max()
    x, _ = cb.get_state()
    assert torch.equal(x, pack(xs).cuda())


def test_bitwise_reproducible():
    cfg, xs, vs, tgs, _ = windows(B=2, n=12, S=3, seed=105)
    w = weights(106)
    tg = targets_of(tgs, 3, 2)
    outs = []
    for _ in range(2):
        cb = ClothBatch(cfg["specs"], cfg["pins"])
        cb.set_state(pack(xs).cuda(), pack(vs).cuda())
        outs.append(cb.train_loss_pcell(w, 3, tg))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_adam_steps_reduce_the_loss():
    cfg, xs, vs, tgs, _ = windows(B=4, n=12, S=3, seed=107)
    tg = targets_of(tgs, 3, 4)
    w = torch.from_numpy(weights(108)).cuda()
    m = torch.zeros(39, device="cuda")
    v = torch.zeros(39, device="cuda")
    cb = ClothBatch(cfg["specs"], cfg["pins"])
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    losses = []
    for t in range(1, 41):
        loss, g = cb.train_loss_pcell(w, 3, tg)
        losses.append(loss.item())
        adam_step(w, g, m, v, t, lr=2e-2 * float(w[:39].abs().mean()), n=39)
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
