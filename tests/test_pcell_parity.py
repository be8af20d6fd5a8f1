"""The literal cell (Eq. 6-7, Fig. 1) and its network step on the GPU vs the
FP64 oracle.

Tolerances: cell output <= 1e-5 normwise per cloth (FP32 differences and
ISRU); positions after 20 network steps <= 1e-4 m.  Ragged batches cover
single nodes, thin strips, sizes off the 32 x 8 tile and several tiles.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack

pytestmark = pytest.mark.gpu

A_TOL = 1e-5
X_TOL = 1e-4


def normwise(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-30))


def batch(seed, shapes, sphere=False, p_sigma=0.5):
    rng = np.random.default_rng(seed)
    specs, pins, xs, vs = [], [], [], []
    for (r, c) in shapes:
        sph = None
        if sphere:
            w = (c - 1) * wl.H_DEFAULT
            sph = {"center": (w / 2, (r - 1) * wl.H_DEFAULT / 2, -0.3 * w - 0.004), "radius": 0.3 * w + 0.005}
        s = wl.cloth_spec(r, c, p=rng.normal(0, p_sigma), sphere=sph)
        x, v = wl.sag_state(s, rng, amp=0.01, vamp=0.1)
        n = r * c
        pins.append(sorted(set(int(i) for i in rng.choice(n, size=min(n, 2), replace=False))) if n > 2 else [])
        specs.append(s); xs.append(x); vs.append(v)
    return specs, pins, xs, vs


SHAPES = [(1, 1), (1, 2), (2, 1), (3, 3), (5, 7), (8, 32), (9, 33), (37, 121), (64, 100)]


def test_cell_output_matches_oracle():
    specs, pins, xs, vs = batch(81, SHAPES)
    w = wl.pcell_blob(82)
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    a = cb.pcell_accel(w)
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(a)]
    for b, s in enumerate(specs):
        ref = oracle.pcell_accel(w.astype(np.float64), s, xs[b].astype(np.float64), vs[b].astype(np.float64))
        assert normwise(got[b], ref) <= A_TOL, (b, s["rows"], s["cols"], normwise(got[b], ref))
    # the state is untouched
    x, v = cb.get_state()
    assert torch.equal(x, pack(xs).cuda())


def test_random_weights_all_branches():
    """Weights of one scale in every branch (the nonlinear and derivative
    branches carry as much as the linear one)."""
    specs, pins, xs, vs = batch(83, [(12, 40), (33, 17)])
    rng = np.random.default_rng(84)
    w = np.concatenate([rng.normal(0, 1e4, 36), [0.3, -0.2, -9.81], [625.0]]).astype(np.float32)
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(cb.pcell_accel(w))]
    for b, s in enumerate(specs):
        ref = oracle.pcell_accel(w.astype(np.float64), s, xs[b].astype(np.float64), vs[b].astype(np.float64))
        assert normwise(got[b], ref) <= A_TOL


@pytest.mark.parametrize("sphere", [False, True])
def test_network_step_matches_oracle(sphere):
    specs, pins, xs, vs = batch(85, [(1, 1), (3, 3), (9, 33), (20, 45)], sphere=sphere)
    w = wl.pcell_blob(86)
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    cb.step_pcell(w, 20)
    x, _ = cb.get_state()
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(x)]
    for b, s in enumerate(specs):
        xr, _ = oracle.pcell_step(w.astype(np.float64), s, xs[b], vs[b], pins=pins[b], steps=20)
        assert np.abs(got[b] - xr).max() <= X_TOL, (b, np.abs(got[b] - xr).max())
    assert cb.status() == 0


def test_zero_rest_length_springs_move_like_the_oracle_springs():
    """w_L = k / m, other branches 0, b_L = g: the cell is Hooke's law with
    zero rest length; 10 steps on the GPU against the oracle's cell."""
    s = wl.cloth_spec(16, 24)
    rng = np.random.default_rng(87)
    x0, v0 = wl.sag_state(s, rng, amp=0.005, vamp=0.0)
    w = np.zeros(40, dtype=np.float32)
    w[0:4], w[4:8], w[8:12] = s["k_struct"] / s["m"], s["k_shear"] / s["m"], s["k_bend"] / s["m"]
    w[36:39] = s["g"]
    w[39] = 1.0
    cb = ClothBatch([s], [[0, 23]])
    cb.set_state(pack([x0]).cuda(), pack([v0]).cuda())
    cb.step_pcell(w, 10)
    x, _ = cb.get_state()
    xr, _ = oracle.pcell_step(w.astype(np.float64), s, x0, v0, pins=[0, 23], steps=10)
    assert np.abs(x.cpu().numpy().reshape(xr.shape) - xr).max() <= X_TOL


def test_step_is_deterministic_and_pins_hold():
    specs, pins, xs, vs = batch(88, [(30, 61), (7, 9)])
    w = wl.pcell_blob(89)
    outs = []
    for _ in range(2):
        cb = ClothBatch(specs, pins)
        cb.set_state(pack(xs).cuda(), pack(vs).cuda())
        cb.step_pcell(w, 15)
        outs.append(cb.get_state())
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    x = outs[0][0].cpu().numpy()
    x0 = pack(xs).numpy()
    for b in range(len(specs)):
        off = sum(s["rows"] * s["cols"] for s in specs[:b])
        for p in pins[b]:
            assert np.array_equal(x[off + p], x0[off + p])
