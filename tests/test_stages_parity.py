"""Training stages on the GPU (Sec. 3.2.1, Table 1, Sec. 5): the Eq. 8 loss
alone (the pre-process objective) equals the loss of the full call; the
masked Adam kernel against the oracle; the trainer's frozen groups and
schedule; the differential-evolution pre-process with libcloth's loss,
its best loss checked by the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import stages
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import FP32, Net, adam_step

pytestmark = pytest.mark.gpu


def windows(B=3, n=10, S=3, seed=301):
    cfg = wl.plain_batch(seed=seed, count=B, side_lo=n, side_hi=n)
    rng = np.random.default_rng(seed + 1)
    xs, vs, tgs, ats = [], [], [], []
    for b in range(B):
        s = cfg["specs"][b]
        x0, v0 = wl.sag_state(s, rng, amp=0.02, vamp=0.05)
        x0 = x0.astype(np.float32).astype(np.float64)
        v0 = v0.astype(np.float32).astype(np.float64)
        tg, xt, vt = [], x0, v0
        for _ in range(S):
            xt, vt = oracle.step(s, xt, vt, pins=cfg["pins"][b], steps=1)
            tg.append(xt.astype(np.float32).astype(np.float64))
        xs.append(x0); vs.append(v0); tgs.append(np.array(tg))
        ats.append((oracle.total_force(s, x0, v0) - oracle.pressure_force(s, x0)) / s["m"])
    targets = torch.from_numpy(np.stack([np.concatenate([tgs[b][t].reshape(-1, 3) for b in range(B)])
                                         for t in range(S)]).astype(np.float32)).cuda()
    x0t = pack([x.astype(np.float32) for x in xs]).cuda()
    v0t = pack([v.astype(np.float32) for v in vs]).cuda()
    return cfg, xs, vs, tgs, ats, targets, x0t, v0t


def oracle_loss(w, cell, cfg, xs, vs, tgs, ats, alpha=0.5, g=9.81):
    B = len(xs)
    tot = 0.0
    for b, s in enumerate(cfg["specs"]):
        l, _ = oracle.unroll_loss(np.asarray(w, dtype=np.float64), s, cfg["pins"][b], xs[b], vs[b], tgs[b], ats[b],
                                  alpha, g, s["h"], with_grad=False, cell=cell)
        tot += l / B
    return tot


def pcell_weights(seed=303):
    rng = np.random.default_rng(seed)
    w = wl.pcell_blob(seed).astype(np.float64)
    w[12:36] *= rng.uniform(0.5, 2.0, 24)
    return w.astype(np.float32)


def cnn_weights(h):
    return wl.kaiming_blob(2011, in_scale=(1.0 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3).astype(np.float32)


def test_loss_alone_equals_the_full_call():
    cfg, xs, vs, tgs, ats, tg, x0, v0 = windows()
    S = tg.shape[0]
    cb = ClothBatch(cfg["specs"], cfg["pins"])
    cb.set_state(x0, v0)
    w = pcell_weights()
    l_full, _ = cb.train_loss_pcell(w, S, tg)
    l_only, g = cb.train_loss_pcell(w, S, tg, with_grad=False)
    assert g is None and torch.equal(l_full, l_only)
    net = Net(cnn_weights(cfg["specs"][0]["h"]), FP32)
    l_full, _ = cb.train_loss(net, S, tg)
    l_only, g = cb.train_loss(net, S, tg, with_grad=False)
    assert g is None and torch.equal(l_full, l_only)
    x, v = cb.get_state()
    assert torch.equal(x, x0) and torch.equal(v, v0)
    cb.close(); net.close()


def test_masked_adam_matches_the_oracle():
    rng = np.random.default_rng(5)
    n = 13027
    th, g = rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32)
    m, v = (rng.normal(size=n) * 0.01).astype(np.float32), (rng.random(n) * 0.01).astype(np.float32)
    mask = stages.freeze_mask("cnn", ["WL", "WN", "bL"], n)
    T = [torch.from_numpy(a.copy()).cuda() for a in (th, g, m, v)]
    adam_step(T[0], T[1], T[2], T[3], t=3, lr=1e-3, n=n, mask=torch.from_numpy(mask).cuda())
    f = lambda a: float(np.float32(a))   # the kernel's float32 hyper-parameters, exactly
    rt, rm, rv = oracle.adam_step_masked(th, g, m, v, t=3, lr=f(1e-3), mask=mask.astype(bool), beta1=f(0.9),
                                         beta2=f(0.999), eps=f(1e-8))
    k = mask.astype(bool)
    got = [a.cpu().numpy() for a in (T[0], T[2], T[3])]
    for a, r, a0 in zip(got, (rt, rm, rv), (th, m, v)):
        assert np.array_equal(a[~k], a0[~k])
        assert np.abs(a[k] - r[k]).max() <= 1e-6 * max(np.abs(r[k]).max(), 1e-30)


def test_trainer_freezes_groups_and_takes_the_scheduled_rate():
    from paper_2403_12820_gb300.train import Dataset, Trainer

    data = Dataset(count=6, n=12, steps=12, seed=1004)
    tr = Trainer(data, batch=3, unroll=3, cell="pcell", trainable=["L_near", "b_L"],
                 lr_schedule=stages.StepLR(2e-3, 1, 0.0))       # 2e-3 at iteration 0, then 0
    w0 = tr.w.clone()
    tr.step()
    w1 = tr.w.clone()
    k = torch.from_numpy(stages.freeze_mask("pcell", ["L_near", "b_L"], 40).astype(bool)).cuda()
    assert torch.equal(w1[~k], w0[~k])
    assert not torch.equal(w1[k], w0[k])
    m1 = tr.m.clone()
    tr.step()                                                    # lr 0: weights stay, moments move
    assert torch.equal(tr.w, w1) and not torch.equal(tr.m, m1)
    tr.set_trainable(None)
    tr.lr_schedule = stages.CosineLR(1e-3, 0.0, 10)
    tr.step()
    assert not torch.equal(tr.w[~k][:36], w1[~k][:36])


@pytest.mark.parametrize("cell", ["pcell", "cnn"])
def test_de_preprocess_with_the_gpu_loss_checked_by_the_oracle(cell):
    if cell == "pcell":
        cfg, xs, vs, tgs, ats, tg, x0, v0 = windows(B=3, n=10, S=3)
        w0, pop, gens = pcell_weights(), 8, 3
    else:
        cfg, xs, vs, tgs, ats, tg, x0, v0 = windows(B=2, n=8, S=2, seed=311)
        w0, pop, gens = cnn_weights(cfg["specs"][0]["h"]), 4, 1
    obj = stages.WindowLoss(cell, w0, cfg["specs"], cfg["pins"], x0, v0, tg)
    draws = wl.de_draws(seed=2007, pop=pop, dim=6, generations=gens)
    res = stages.de_preprocess(obj, draws, bounds=(-3.0, 3.0))
    assert res["evals"] == pop * (gens + 1) == obj.calls
    l0 = obj.loss_of_blob(w0)                     # member 0 started at the unscaled blob
    obj.close()
    assert all(b <= a for a, b in zip(res["history"], res["history"][1:]))
    assert res["f"] <= l0
    f1 = oracle_loss(w0, cell, cfg, xs, vs, tgs, ats)
    assert abs(l0 - f1) <= 1e-4 * abs(f1), (l0, f1)
    fb = oracle_loss(res["blob"], cell, cfg, xs, vs, tgs, ats)
    assert abs(res["f"] - fb) <= 1e-4 * abs(fb), (res["f"], fb)
    ref = oracle.scaled_blob(w0.astype(np.float64), cell, res["x"])
    assert np.array_equal(res["blob"], ref.astype(np.float32))


def test_trainer_pre_process_applies_the_scales():
    from paper_2403_12820_gb300.train import Dataset, Trainer

    data = Dataset(count=6, n=12, steps=12, seed=1004)
    tr = Trainer(data, batch=3, unroll=3, cell="pcell")
    tr.step()
    res = tr.pre_process(wl.de_draws(seed=5, pop=6, dim=6, generations=2))
    assert tr.t == 0 and float(tr.m.abs().sum()) == 0.0
    assert np.array_equal(tr.w.cpu().numpy(), res["blob"])
    assert res["groups"] == ["L_near", "L_far", "N_near", "N_far", "D_near", "D_far"]
    assert np.isfinite(res["f"])
