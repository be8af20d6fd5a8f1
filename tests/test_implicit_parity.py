"""Implicit plain step on the GPU (linearised backward Euler, matrix-free CG)
vs the FP64 oracle's direct solve of the same linear system: positions
within 1e-4 m and velocities within 1e-3 normwise (cloths without a
sphere, whose contact stops a node on whichever side of the surface the
rounding puts it) after several steps of
stride x dt (pins moving, pressure, drag, sphere contact with and without
friction); bitwise reproducible; zero CG iterations leave the free
velocities as they are."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import _lib
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack

pytestmark = pytest.mark.gpu


def batch(seed, shapes):
    rng = np.random.default_rng(seed)
    specs, pins, xs, vs = [], [], [], []
    for i, (r, c) in enumerate(shapes):
        w = (c - 1) * wl.H_DEFAULT
        sph = ({"center": (w / 2, (r - 1) * wl.H_DEFAULT / 2, -0.3 * w - 0.004), "radius": 0.3 * w + 0.005,
                "friction": (-1.0, 0.3)[i % 2]} if i % 3 == 1 else None)
        s = wl.cloth_spec(r, c, p=rng.normal(0, 0.5), sphere=sph, pin_v=rng.normal(0, 0.05, 3) if i % 2 else None)
        x, v = wl.sag_state(s, rng, amp=0.01, vamp=0.05)
        n = r * c
        pins.append(sorted(set(int(k) for k in rng.choice(n, size=min(n, 3), replace=False))) if n > 2 else [])
        specs.append(s); xs.append(x); vs.append(v)
    return specs, pins, xs, vs


def normwise(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-30))


@pytest.mark.parametrize("stride", [1, 4, 10])
def test_matches_the_oracle_direct_solve(stride):
    specs, pins, xs, vs = batch(701, [(1, 1), (3, 3), (9, 33), (20, 45), (16, 130)])
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    cb.step_implicit(3, stride=stride, cg_iters=80)
    x, v = cb.get_state()
    gx = [t.cpu().numpy().astype(np.float64) for t in cb.split(x)]
    gv = [t.cpu().numpy().astype(np.float64) for t in cb.split(v)]
    for b, s in enumerate(specs):
        xr, vr = oracle.implicit_step(s, xs[b].astype(np.float64), vs[b].astype(np.float64), pins=pins[b], steps=3,
                                      stride=stride)
        assert np.abs(gx[b] - xr).max() <= 1e-4, (b, np.abs(gx[b] - xr).max())
        if "sphere" not in s:   # a contact decision taken either side of the surface stops a node or not
            assert normwise(gv[b], vr) <= 1e-3, (b, normwise(gv[b], vr))
    assert cb.status() == 0
    cb.close()


def test_bitwise_reproducible_and_state_untouched_by_zero_steps():
    specs, pins, xs, vs = batch(703, [(9, 33), (40, 41)])
    outs = []
    for _ in range(2):
        cb = ClothBatch(specs, pins)
        cb.set_state(pack(xs).cuda(), pack(vs).cuda())
        cb.step_implicit(0, stride=5)
        x0, _ = cb.get_state()
        assert torch.equal(x0, pack(xs).cuda())
        cb.step_implicit(4, stride=5, cg_iters=15)
        outs.append(cb.get_state())
        cb.close()
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_zero_iterations_keep_the_free_velocities():
    specs, pins, xs, vs = batch(705, [(9, 33)])
    specs = [dict(specs[0])]
    specs[0].pop("sphere", None)
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    cb.step_implicit(1, stride=3, cg_iters=0)
    x, v = cb.get_state()
    free = ~oracle.pin_mask(specs[0], pins[0]).astype(bool)
    v0 = vs[0].reshape(-1, 3)
    assert np.array_equal(v.cpu().numpy()[free], v0[free].astype(np.float32))
    h = np.float32(3 * specs[0]["dt"])
    want = xs[0].reshape(-1, 3)[free].astype(np.float32) + h * v0[free].astype(np.float32)
    assert np.abs(x.cpu().numpy()[free] - want).max() <= 1e-6
    cb.close()


def test_rejects_bad_arguments():
    specs, pins, xs, vs = batch(707, [(3, 3)])
    cb = ClothBatch(specs, pins)
    for args in ((-1, 1, 10), (1, 0, 10), (1, 1001, 10), (1, 1, -1)):
        with pytest.raises(_lib.ClothError):
            cb.step_implicit(*args[:1], stride=args[1], cg_iters=args[2])
    cb.close()
