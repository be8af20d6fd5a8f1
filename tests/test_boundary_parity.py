"""Moving pins and friction contact on the GPU vs the FP64 oracle (Sec. 3.1:
the cloth part that moves along with another object, intersection
elimination with dry friction; Sec. 3.2: boundary treatments selectable at
run time).  Every step kernel — the plain step (with and without spring-axis
damping), the FP32 and BF16 network steps, the literal cell — takes the pin
velocity and the Coulomb contact from the cloth's descriptor; positions
after the steps within 1e-4 m of the oracle, the Eq. 8 loss and gradient
with moving pins within 1e-4."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import _lib
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import BF16, FP32, Net

pytestmark = pytest.mark.gpu

X_TOL = 1e-4
FRICTIONS = (-1.0, 0.0, 0.3, 2.0)


def batch(seed, shapes, mu=0.0):
    """Cloths sagging onto a sphere under their middle (1 mm of overlap at
    the start), pins moving with per-cloth velocities, each contact model."""
    rng = np.random.default_rng(seed)
    specs, pins, xs, vs = [], [], [], []
    for i, (r, c) in enumerate(shapes):
        w = (c - 1) * wl.H_DEFAULT
        sph = {"center": (w / 2, (r - 1) * wl.H_DEFAULT / 2, -0.3 * w - 0.004), "radius": 0.3 * w + 0.005,
               "friction": FRICTIONS[i % len(FRICTIONS)]}
        s = wl.cloth_spec(r, c, p=rng.normal(0, 0.5), sphere=sph, mu=mu, pin_v=rng.normal(0, 0.2, 3))
        x, v = wl.sag_state(s, rng, amp=0.01, vamp=0.1)
        n = r * c
        pins.append(sorted(set(int(k) for k in rng.choice(n, size=min(n, 3), replace=False))) if n > 2 else [])
        specs.append(s); xs.append(x); vs.append(v)
    return specs, pins, xs, vs


def compare(cb, specs, step_fn, xs, vs, pins, steps):
    x, _ = cb.get_state()
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(x)]
    for b, s in enumerate(specs):
        xr, _ = step_fn(s, xs[b].astype(np.float64), vs[b].astype(np.float64), pins[b], steps)
        err = np.abs(got[b] - xr).max()
        assert err <= X_TOL, (b, s["rows"], s["cols"], s["sphere"]["friction"], err)
    assert cb.status() == 0


SHAPES = [(3, 3), (9, 33), (20, 45), (16, 130), (33, 64), (7, 7), (40, 41), (12, 250)]


@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_plain_step(mu):
    specs, pins, xs, vs = batch(501, SHAPES, mu=mu)
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    cb.rollout(100, graph_chunk=20)
    compare(cb, specs, lambda s, x, v, p, k: oracle.step(s, x, v, pins=p, steps=k), xs, vs, pins, 100)
    cb.close()


def test_plain_step_pins_travel_with_their_object():
    """Away from the sphere a pinned node moves by exactly dt * pin_v per step
    (in float32, up to the rounding of the 100 additions)."""
    specs, pins, xs, vs = batch(502, [(9, 33), (20, 45)])
    specs = [dict(s) for s in specs]
    for s in specs:
        del s["sphere"]
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    cb.rollout(100, graph_chunk=20)
    x, v = cb.get_state()
    for b, (s, xb, vb) in enumerate(zip(specs, cb.split(x), cb.split(v))):
        xb = xb.cpu().numpy().reshape(-1, 3)[pins[b]]
        want = xs[b].reshape(-1, 3)[pins[b]] + 100 * s["dt"] * np.asarray(s["pin_v"], dtype=np.float32)
        assert np.abs(xb - want).max() <= 1e-6
        assert np.array_equal(vb.cpu().numpy().reshape(-1, 3)[pins[b]],
                              np.broadcast_to(np.asarray(s["pin_v"], dtype=np.float32), (len(pins[b]), 3)))
    cb.close()


def blob(seed, h=wl.H_DEFAULT):
    return wl.kaiming_blob(seed, in_scale=(1.0 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.0)


@pytest.mark.parametrize("precision", [FP32, BF16])
def test_network_step(precision):
    specs, pins, xs, vs = batch(503, [(5, 7), (16, 33), (30, 61), (12, 28)])
    w = blob(504)
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    net = Net(w, precision)
    cb.step_net(net, 20)
    compare(cb, specs, lambda s, x, v, p, k: oracle.net_step(w.astype(np.float64), s, x, v, pins=p, steps=k),
            xs, vs, pins, 20)
    cb.close(); net.close()


def test_literal_cell_step():
    specs, pins, xs, vs = batch(505, [(1, 1), (3, 3), (9, 33), (20, 45)])
    w = wl.pcell_blob(506)
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    cb.step_pcell(w, 20)
    compare(cb, specs, lambda s, x, v, p, k: oracle.pcell_step(w.astype(np.float64), s, x, v, pins=p, steps=k),
            xs, vs, pins, 20)
    cb.close()


def test_boundary_selected_between_graph_replays():
    """The same cached graph before and after cloth_set_boundary: the kernels
    read the new pin velocity and friction from the descriptors."""
    specs, pins, xs, vs = batch(507, [(9, 33), (20, 45), (16, 130)])
    fixed = [dict(s, pin_v=(0.0, 0.0, 0.0), sphere=dict(s["sphere"], friction=-1.0)) for s in specs]
    cb = ClothBatch(fixed, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    cb.rollout(40, graph_chunk=20)
    for b, s in enumerate(specs):
        cb.set_boundary(b, s["pin_v"], s["sphere"]["friction"])
    cb.rollout(40, graph_chunk=20)

    def two_phase(b, x, v, p):
        x, v = oracle.step(fixed[b], x, v, pins=p, steps=40)
        return oracle.step(specs[b], x, v, pins=p, steps=40)

    x, _ = cb.get_state()
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(x)]
    for b in range(len(specs)):
        xr, _ = two_phase(b, xs[b].astype(np.float64), vs[b].astype(np.float64), pins[b])
        assert np.abs(got[b] - xr).max() <= X_TOL, b
    with pytest.raises(_lib.ClothError):
        cb.set_boundary(0, (float("nan"), 0.0, 0.0), -1.0)
    with pytest.raises(_lib.ClothError):
        cb.set_boundary(3, (0.0, 0.0, 0.0), -1.0)
    cb.close()


def test_training_loss_with_moving_pins():
    S, alpha, g = 3, 0.5, 9.81
    cfg = wl.plain_batch(seed=509, count=3, side_lo=10, side_hi=10)
    rng = np.random.default_rng(510)
    specs, xs, vs, tgs, ats = [], [], [], [], []
    for b in range(3):
        s = dict(cfg["specs"][b], pin_v=[wl.f32(a) for a in rng.normal(0, 0.1, 3)])
        x0, v0 = wl.sag_state(s, rng, amp=0.02, vamp=0.05)
        x0 = x0.astype(np.float32).astype(np.float64)
        v0 = v0.astype(np.float32).astype(np.float64)
        tg, xt, vt = [], x0, v0
        for _ in range(S):
            xt, vt = oracle.step(s, xt, vt, pins=cfg["pins"][b], steps=1)
            tg.append(xt.astype(np.float32).astype(np.float64))
        specs.append(s); xs.append(x0); vs.append(v0); tgs.append(np.array(tg))
        ats.append((oracle.total_force(s, x0, v0) - oracle.pressure_force(s, x0)) / s["m"])
    rng_w = np.random.default_rng(511)
    w = wl.pcell_blob(511).astype(np.float64)
    w[12:36] *= rng_w.uniform(0.5, 2.0, 24)
    w = w.astype(np.float32)
    rl, rg = 0.0, np.zeros(40)
    for b, s in enumerate(specs):
        l, gw = oracle.unroll_loss(w.astype(np.float64), s, cfg["pins"][b], xs[b], vs[b], tgs[b], ats[b], alpha, g,
                                   s["h"], cell="pcell")
        rl += l / 3; rg += gw / 3
    cb = ClothBatch(specs, cfg["pins"])
    cb.set_state(pack([x.astype(np.float32) for x in xs]).cuda(), pack([v.astype(np.float32) for v in vs]).cuda())
    tg = torch.from_numpy(np.stack([np.concatenate([tgs[b][t].reshape(-1, 3) for b in range(3)])
                                    for t in range(S)]).astype(np.float32)).cuda()
    loss, grad = cb.train_loss_pcell(w, S, tg, alpha=alpha, g_norm=g)
    assert abs(loss.item() - rl) <= 1e-4 * abs(rl), (loss.item(), rl)
    gg = grad.cpu().numpy()
    assert np.abs(gg[:39] - rg[:39]).max() <= 1e-4 * np.abs(rg[:39]).max()
    cb.close()


def test_plain_step_with_more_pins_than_the_pin_list_holds():
    """The undamped plain step sets its pinned nodes after the step, from the
    context's pin list, or from the pin mask when a context has more pins
    than the list holds (one per 32 nodes): a batch with every boundary node
    of a 40 x 40 cloth pinned (156 pins, moving), beside cloths with a few
    pins, against the oracle after 20 steps; and the same cloths in a batch
    whose pins fit the list."""
    specs, pins, xs, vs = batch(311, [(40, 40), (9, 33), (21, 6)])
    pins[0] = [int(k) for k in wl.boundary_nodes(40, 40)]
    for sel in ([0, 1, 2], [1, 2]):
        sp, pn = [specs[i] for i in sel], [pins[i] for i in sel]
        cb = ClothBatch(sp, pn)
        cb.set_state(pack([xs[i] for i in sel]).cuda(), pack([vs[i] for i in sel]).cuda())
        cb.step(20)
        x, v = cb.get_state()
        got = [t.cpu().numpy().astype(np.float64) for t in cb.split(x)]
        gotv = [t.cpu().numpy().astype(np.float64) for t in cb.split(v)]
        for j, i in enumerate(sel):
            xr, vr = oracle.step(specs[i], xs[i], vs[i], pins=pins[i], steps=20)
            assert np.abs(got[j] - xr).max() <= X_TOL, (sel, i)
            assert np.abs(gotv[j] - vr).max() <= 1e-2, (sel, i)
        assert cb.status() == 0
        cb.close()
