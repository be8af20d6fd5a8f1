"""Launch-shape autotuner of the plain step: the host logic (candidates, cache
keys, the JSON cache, the choice of the fastest) on the CPU, and the timing
entry point cloth_tune_launch on the GPU (the state does not move, the
fastest shape is applied, results do not depend on it)."""
import json

import numpy as np
import pytest

from paper_2403_12820_gb300 import tune


def test_validate_accepts_the_set_launch_ranges():
    assert tune.validate([(4, -1), (-1, 64), (100, 1)]) == [(4, -1), (-1, 64), (100, 1)]
    assert tune.validate(tune.DEFAULT_CANDIDATES) == list(tune.DEFAULT_CANDIDATES)
    for bad in ([(3, -1)], [(0, -1)], [(-2, -1)], [(8, 0)], [(8, 65)], [(8, -2)], []):
        with pytest.raises(ValueError):
            tune.validate(bad)


def test_batch_key_separates_what_the_work_list_depends_on():
    g = [(64, 64), (100, 37)]
    k = tune.batch_key("plain_step", "GB300", 152, g)
    assert k == tune.batch_key("plain_step", "GB300", 152, [(64, 64), (100, 37)])
    assert k == tune.batch_key("plain_step", "GB300", 152, np.array(g))
    others = [tune.batch_key("plain_step_damp", "GB300", 152, g), tune.batch_key("plain_step", "B200", 152, g),
              tune.batch_key("plain_step", "GB300", 148, g), tune.batch_key("plain_step", "GB300", 152, g[::-1]),
              tune.batch_key("plain_step", "GB300", 152, [(64, 64), (100, 38)]),
              tune.batch_key("plain_step", "GB300", 152, g[:1])]
    assert len(set(others + [k])) == len(others) + 1
    assert k.startswith("plain_step/152sm/2x/")


def test_kernel_name_follows_the_damping():
    assert tune.kernel_name([{"mu": 0.0}, {}]) == "plain_step"
    assert tune.kernel_name([{"mu": 0.0}, {"mu": 0.02}]) == "plain_step_damp"


def test_pick_takes_the_first_fastest():
    c = [(8, -1), (16, -1), (-1, -1)]
    assert tune.pick(c, [3.0, 2.0, 2.5]) == 1
    assert tune.pick(c, [2.0, 2.0, 2.0]) == 0
    with pytest.raises(ValueError):
        tune.pick(c, [1.0, 2.0])


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "launch.json")
    c = tune.LaunchCache(path)
    assert c.get("a") is None
    rec = {"seg_rows": 32, "warps_per_sm": -1, "us_per_step": 74.2, "candidates": [[32, -1, 74.2]]}
    c.put("a", rec)
    c.put("b", dict(rec, seg_rows=-1, warps_per_sm=16))
    again = tune.LaunchCache(path)
    assert again.get("a") == rec and again.get("b")["warps_per_sm"] == 16
    with open(path) as fh:
        assert set(json.load(fh)) == {"a", "b"}


def test_cache_rejects_bad_files(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("[1, 2]")
    with pytest.raises(ValueError):
        tune.LaunchCache(str(p))
    p.write_text(json.dumps({"k": {"seg_rows": 2, "warps_per_sm": -1}}))
    with pytest.raises(ValueError):
        tune.LaunchCache(str(p)).get("k")


# --------------------------------------------------------------------- GPU


def _batch():
    from paper_2403_12820_gb300 import workloads as wl
    from paper_2403_12820_gb300.cloth import ClothBatch, pack

    rng = np.random.default_rng(41)
    specs, pins, xs, vs = [], [], [], []
    for (r, c) in [(3, 3), (37, 121), (130, 250), (64, 64), (9, 241), (200, 130)]:
        s = wl.cloth_spec(r, c, k=(500.0, 250.0, 50.0), p=float(rng.normal(0, 0.5)), drag=0.01)
        x, v = wl.sag_state(s, rng, amp=0.02, vamp=0.1)
        specs.append(s); xs.append(x); vs.append(v)
        pins.append([0, c - 1] if r * c > 2 else [])
    cb = ClothBatch(specs, pins)
    x0, v0 = pack(xs).cuda(), pack(vs).cuda()
    cb.set_state(x0, v0)
    return cb, x0, v0


@pytest.mark.gpu
def test_tuning_leaves_the_state_and_applies_the_fastest(tmp_path):
    import torch

    cb, x0, v0 = _batch()
    cands = [(4, -1), (16, -1), (-1, -1), (-1, 4), (32, 12)]
    rec = tune.autotune(cb, cache_path=str(tmp_path / "l.json"), candidates=cands, warmup=2, steps=5)
    assert not rec["cached"] and len(rec["candidates"]) == len(cands)
    assert all(t > 0 for (_, _, t) in rec["candidates"])
    i = tune.pick(cands, [t for (_, _, t) in rec["candidates"]])
    assert (rec["seg_rows"], rec["warps_per_sm"]) == cands[i]
    seg, w, _ = cb.get_launch()
    assert seg == (cands[i][0] if cands[i][0] > 0 else 0) and w == (cands[i][1] if cands[i][1] > 0 else 0)
    x, v = cb.get_state()
    assert torch.equal(x, x0) and torch.equal(v, v0), "tuning moved the state"
    assert cb.status() == 0
    # the tuned shape steps to the same bits as the default shape
    cb.step(10)
    xt, vt = cb.get_state()
    ref, _, _ = _batch()
    ref.step(10)
    xr, vr = ref.get_state()
    assert torch.equal(xt, xr) and torch.equal(vt, vr)
    # a second batch of the same shape takes the cached shape without timing
    cb2, _, _ = _batch()
    rec2 = tune.autotune(cb2, cache_path=str(tmp_path / "l.json"), candidates=cands)
    assert rec2["cached"] and rec2["key"] == rec["key"]
    assert cb2.get_launch()[:2] == cb.get_launch()[:2]
    for c in (cb, cb2, ref):
        c.close()


@pytest.mark.gpu
def test_tune_rejects_bad_candidates_before_running():
    from paper_2403_12820_gb300 import _lib

    cb, _, _ = _batch()
    before = cb.get_launch()
    with pytest.raises(_lib.ClothError):
        cb.tune_launch([(16, -1), (2, -1)])
    with pytest.raises(_lib.ClothError):
        cb.tune_launch([(16, 70)])
    with pytest.raises(_lib.ClothError):
        cb.tune_launch([(16, -1)], steps=0)
    assert cb.get_launch() == before
    cb.close()


def test_net_tile_choices_are_the_library_shapes():
    """The network step's tile shapes per precision (host query, no GPU):
    FP32 has the tensor-core three-term shapes of 10 and 6 rows (the default
    first) and then the CUDA-core shapes of 14 rows; BF16 has tensor-core
    shapes of 14, 10 and 6 rows; every shape distinct."""
    from paper_2403_12820_gb300.net import BF16, FP32
    f = tune.net_tile_choices(FP32)
    assert f[:2] == [{"rows": r, "cols": 26, "kind": "tensor"} for r in (10, 6)]
    assert f[2] == {"rows": 14, "cols": 14, "kind": "cuda"}
    assert [c["kind"] for c in f[2:]] == ["cuda"] * (len(f) - 2) and len(f) >= 4
    b = tune.net_tile_choices(BF16)
    assert b == [{"rows": r, "cols": 26, "kind": "tensor"} for r in (14, 10, 6)]
    for ch in (f, b):
        assert len({(c["rows"], c["cols"], c["kind"]) for c in ch}) == len(ch)
    with pytest.raises(Exception):
        tune.net_tile_choices(7)


def _uneven_batch(seed):
    """An uneven batch: single nodes, thin strips, sizes off every tile
    shape, pins, pressure, a sphere."""
    from paper_2403_12820_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    specs, pins, xs, vs = [], [], [], []
    for (r, c) in [(1, 1), (1, 7), (5, 3), (14, 14), (15, 31), (29, 61), (40, 13), (70, 33)]:
        sph = {"center": (0.1, 0.1, -0.05), "radius": 0.06} if r == 29 else None
        sp = wl.cloth_spec(r, c, p=rng.normal(0, 0.5), sphere=sph)
        x, v = wl.sag_state(sp, rng, amp=0.02, vamp=0.1)
        specs.append(sp); xs.append(x); vs.append(v); pins.append([0] if r * c > 1 else [])
    return specs, pins, xs, vs


@pytest.mark.gpu
@pytest.mark.parametrize("prec_name", ["fp32", "bf16"])
def test_network_step_per_tile_shape_and_the_tuner_picks_the_fastest(tmp_path, prec_name):
    """Each node's arithmetic does not depend on the tiling, so the shapes of
    one kind give the same state bit for bit; the FP32 tensor-core shape
    (three BF16 products per term) agrees with the CUDA-core ones within the
    FP32 tolerance on the velocity change; cloth_tune_net leaves the state,
    applies the fastest shape, and the cache brings it back without timing."""
    import torch

    from paper_2403_12820_gb300 import workloads as wl
    from paper_2403_12820_gb300.cloth import ClothBatch, pack
    from paper_2403_12820_gb300.net import BF16, FP32, Net
    prec = FP32 if prec_name == "fp32" else BF16
    specs, pins, xs, vs = _uneven_batch(401)
    w = wl.kaiming_blob(402, in_scale=(50.0,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.1)
    net = Net(w, prec)
    x0, v0 = pack(xs).cuda(), pack(vs).cuda()
    choices = tune.net_tile_choices(prec)
    outs = []
    for i, ch in enumerate(choices):
        cb = ClothBatch(specs, pins)
        cb.set_net_tile(prec, i)
        assert cb.get_net_tile(prec) == i
        cb.set_state(x0, v0)
        cb.step_net(net, 1)
        outs.append((ch["kind"], cb.get_state()))
        assert cb.status() == 0
        cb.close()
    ref = [o for k, o in outs if k == outs[0][0]]
    for x, v in ref[1:]:
        assert torch.equal(x, ref[0][0]) and torch.equal(v, ref[0][1])
    for k, (x, v) in outs:
        if k != outs[0][0]:   # the other kind: the velocity change dt * a within the FP32 tolerance
            dv0, dv = (ref[0][1] - v0).double(), (v - v0).double()
            assert float(torch.linalg.norm(dv - dv0) / torch.linalg.norm(dv0)) <= 1e-4
    cb = ClothBatch(specs, pins)
    cb.set_state(x0, v0)
    with pytest.raises(Exception):
        cb.set_net_tile(prec, len(choices))
    path = str(tmp_path / "net_tiles.json")
    rec = tune.autotune_net(cb, net, cache_path=path, warmup=1, steps=3)
    assert not rec["cached"] and rec["shape"] == choices[rec["choice"]]
    assert rec["choice"] == min(range(len(choices)), key=lambda i: rec["candidates"][i][1])
    assert cb.get_net_tile(prec) == rec["choice"]
    x, v = cb.get_state()
    assert torch.equal(x, x0) and torch.equal(v, v0)          # tuning does not move the state
    cb.set_net_tile(prec, 0 if rec["choice"] else 1)
    again = tune.autotune_net(cb, net, cache_path=path)
    assert again["cached"] and cb.get_net_tile(prec) == rec["choice"]
    cb.close()
