"""GPU plain step (libcloth) vs the FP64 oracle, element by element.

Tolerances (normwise = max |gpu - ref| / max |ref| over a cloth):
  forces (Eq. 1-4)            <= 1e-5 normwise, at the seeded start state
                                 and at a strained state
  positions after 200 steps   <= 1e-4 m max abs
  topology                    bit-exact
Inputs are float32; the oracle receives their exact float64 promotions.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
X_TOL = 1e-4


def make(specs, pins, xs, vs):
    cb = ClothBatch(specs, pins)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    return cb


def normwise(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-30))


def per_cloth(cb, t):
    return [a.cpu().numpy().astype(np.float64) for a in cb.split(t)]


def uneven_batch(seed=7, mu=0.0, with_pressure=True):
    """Ragged shapes: single nodes, thin strips, sizes not a multiple of 4,
    several 120-column strips with a tail, rows fewer than a segment."""
    rng = np.random.default_rng(seed)
    shapes = [(1, 1), (1, 2), (2, 1), (3, 3), (5, 7), (16, 33), (37, 121), (130, 250), (9, 241)]
    specs, pins, xs, vs = [], [], [], []
    for (r, c) in shapes:
        s = wl.cloth_spec(r, c, k=(500 * rng.uniform(0.8, 1.2), 250.0, 50.0), mu=mu,
                          p=rng.normal(0, 0.5) if with_pressure else 0.0, drag=0.01)
        x, v = wl.sag_state(s, rng, amp=0.02, vamp=0.1)
        n = r * c
        pins.append(sorted(set(int(i) for i in rng.choice(n, size=min(n, 3), replace=False))) if n > 2 else [])
        specs.append(s); xs.append(x); vs.append(v)
    return specs, pins, xs, vs


def check_forces(specs, pins, xs, vs):
    cb = make(specs, pins, xs, vs)
    got = per_cloth(cb, cb.forces())
    for b, s in enumerate(specs):
        ref = oracle.total_force(s, xs[b].astype(np.float64), vs[b].astype(np.float64))
        assert normwise(got[b], ref) <= F_TOL, (b, s["rows"], s["cols"], normwise(got[b], ref))
    cb.close()


def test_forces_single_cloth_start_state():
    cfg = wl.single_cloth()
    check_forces(cfg["specs"], cfg["pins"], cfg["x"], cfg["v"])


def test_forces_single_cloth_strained_state():
    cfg = wl.single_cloth()
    s, pins = cfg["specs"][0], cfg["pins"][0]
    x, v = oracle.step(s, cfg["x"][0], cfg["v"][0], pins=pins, steps=200)
    check_forces([s], [pins], [x.astype(np.float32)], [v.astype(np.float32)])


@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_forces_uneven_batch(mu):
    check_forces(*uneven_batch(mu=mu))


def test_positions_single_cloth_200_steps():
    cfg = wl.single_cloth()
    s, pins = cfg["specs"][0], cfg["pins"][0]
    cb = make(cfg["specs"], cfg["pins"], cfg["x"], cfg["v"])
    cb.step(200)
    x, v = cb.get_state()
    xr, vr = oracle.step(s, cfg["x"][0], cfg["v"][0], pins=pins, steps=200)
    err = np.abs(x.cpu().numpy().reshape(xr.shape) - xr).max()
    assert err <= X_TOL, err
    assert cb.status() == 0


@pytest.mark.slow
def test_positions_single_cloth_2000_steps():
    cfg = wl.single_cloth()
    s, pins = cfg["specs"][0], cfg["pins"][0]
    cb = make(cfg["specs"], cfg["pins"], cfg["x"], cfg["v"])
    cb.rollout(2000, graph_chunk=100)
    x, _ = cb.get_state()
    xr, _ = oracle.step(s, cfg["x"][0], cfg["v"][0], pins=pins, steps=2000)
    err = np.abs(x.cpu().numpy().reshape(xr.shape) - xr).max()
    assert err <= X_TOL, err


def test_positions_uneven_batch_200_steps():
    specs, pins, xs, vs = uneven_batch(seed=9)
    cb = make(specs, pins, xs, vs)
    cb.step(200)
    x, _ = cb.get_state()
    got = per_cloth(cb, x)
    for b, s in enumerate(specs):
        xr, _ = oracle.step(s, xs[b], vs[b], pins=pins[b], steps=200)
        assert np.abs(got[b] - xr).max() <= X_TOL, (b, np.abs(got[b] - xr).max())


def test_pinned_nodes_do_not_move():
    specs, pins, xs, vs = uneven_batch(seed=10)
    cb = make(specs, pins, xs, vs)
    cb.step(50)
    x, v = cb.get_state()
    gx, gv = per_cloth(cb, x), per_cloth(cb, v)
    for b in range(len(specs)):
        for p in pins[b]:
            assert np.array_equal(gx[b].reshape(-1, 3)[p], xs[b].reshape(-1, 3)[p].astype(np.float64))
            assert np.all(gv[b].reshape(-1, 3)[p] == 0.0)


def test_sphere_contact_matches_oracle():
    """A cloth dropped onto a sphere just below it (the ball scene, Sec. 3.2.2)."""
    n = 24
    w = (n - 1) * 0.02
    R = 0.3 * w
    s = wl.cloth_spec(n, n, g=(0.0, 0.0, -9.81), sphere={"center": (w / 2, w / 2, -R - 1e-4), "radius": R})
    x, v = wl.noisy_flat_state(s, 1e-5, np.random.default_rng(3))
    v[..., 2] = -0.5
    cb = make([s], [[]], [x], [v])
    cb.step(100)
    xg, vg = cb.get_state()
    xr, vr = oracle.step(s, x, v, steps=100)
    xg = xg.cpu().numpy().reshape(xr.shape)
    assert np.abs(xg - xr).max() <= X_TOL
    d = np.linalg.norm(xr - np.array(s["sphere"]["center"]), axis=2)
    assert (d <= R * (1 + 1e-6)).sum() > 10      # some nodes rest on the sphere


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (4, 4), (7, 5), (33, 130), (128, 128)])
def test_topology_bit_exact(shape):
    r, c = shape
    s = wl.cloth_spec(r, c)
    cb = ClothBatch([s])
    m = cb.topology(0).cpu().numpy().view(np.uint16).reshape(r, c)
    assert np.array_equal(m, oracle.neighbor_mask(r, c))


def test_graph_rollout_and_record_match_single_steps():
    specs, pins, xs, vs = uneven_batch(seed=11)
    a = make(specs, pins, xs, vs)
    b = make(specs, pins, xs, vs)
    a.step(30)
    b.rollout(30, graph_chunk=8)            # 3 graph replays + 6 direct steps
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert torch.equal(xa, xb) and torch.equal(va, vb)
    c = make(specs, pins, xs, vs)
    rec = torch.empty(3, c.total_nodes, 3, device="cuda")
    c.rollout(30, record=rec, record_every=10)
    xc, _ = c.get_state()
    assert torch.equal(xc, xa)
    assert torch.equal(rec[2], xa)


@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_launch_shapes_give_identical_results(mu):
    """Every launch shape (balanced ranges, fixed segments, few or many
    warps) runs the same arithmetic per node: bitwise equal states."""
    specs, pins, xs, vs = uneven_batch(seed=13, mu=mu)
    ref = make(specs, pins, xs, vs)
    assert ref.get_launch()[1] == 0   # default warp count
    ref.step(12)
    xr, vr = ref.get_state()
    for seg, w in [(4, 1), (8, 4), (32, 12), (-1, 1), (-1, 64), (-1, -1), (5, 3), (16, -1)]:
        cb = make(specs, pins, xs, vs)
        cb.set_launch(seg, w)
        cb.step(12)
        x, v = cb.get_state()
        assert torch.equal(x, xr) and torch.equal(v, vr), (seg, w)
        assert cb.status() == 0


def test_bitwise_deterministic():
    specs, pins, xs, vs = uneven_batch(seed=12)
    outs = []
    for _ in range(2):
        cb = make(specs, pins, xs, vs)
        cb.rollout(40, graph_chunk=10)
        outs.append(cb.get_state())
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_nonfinite_state_sets_status():
    cfg = wl.single_cloth()
    x = cfg["x"][0].copy()
    x[5, 5, 2] = np.nan
    cb = make(cfg["specs"], cfg["pins"], [x], cfg["v"])
    cb.step(1)
    assert cb.status(clear=True) & 1
    assert cb.status() == 0


def test_full_size_batch_sampled_against_oracle():
    """The 64-cloth batch (sides 64..512) in the benchmark's launch
    configuration (graph-captured chunks); the smallest, a middle and the
    largest cloth are compared with the oracle after 20 steps."""
    cfg = wl.plain_batch()
    cb = make(cfg["specs"], cfg["pins"], cfg["x"], cfg["v"])
    cb.rollout(20, graph_chunk=10)
    x, _ = cb.get_state()
    got = per_cloth(cb, x)
    sizes = [s["rows"] for s in cfg["specs"]]
    order = np.argsort(sizes)
    for b in (order[0], order[len(order) // 2], order[-1]):
        s = cfg["specs"][b]
        xr, _ = oracle.step(s, cfg["x"][b], cfg["v"][b], pins=cfg["pins"][b], steps=20)
        assert np.abs(got[b] - xr).max() <= X_TOL, (b, sizes[b])
    assert cb.status() == 0


def _window(spec, x, v, r, c, rad):
    """Sub-grid of radius `rad` around node (r, c), clipped at the cloth's
    edges, as its own cloth spec and state; returns (spec, x, v, (r, c) in it)."""
    r0, r1 = max(0, r - rad), min(spec["rows"], r + rad + 1)
    c0, c1 = max(0, c - rad), min(spec["cols"], c + rad + 1)
    s = dict(spec)
    s["rows"], s["cols"] = r1 - r0, c1 - c0
    # the window's lattice starts at (c0 h, r0 h): shift positions so that
    # the rest state of the window is the oracle's lattice
    sh = np.array([c0 * spec["h"], r0 * spec["h"], 0.0])
    return s, x[r0:r1, c0:c1] - sh, v[r0:r1, c0:c1], (r - r0, c - c0), sh


@pytest.mark.parametrize("steps", [1, 3])
def test_maximum_size_cloth_sampled_against_oracle(steps):
    """One 4096 x 4096 cloth (16.8M nodes, 0.8 GB of state): after `steps`
    steps, sampled nodes (corners, edges, interior) equal the oracle run on
    the window of radius 2 * steps around them, which holds every node they
    depend on.  A node pinned and pressure on."""
    n = 4096
    rng = np.random.default_rng(91)
    s = wl.cloth_spec(n, n, p=0.4)
    x, v = wl.noisy_flat_state(s, 1e-4, rng)
    pins = [0, n - 1]
    cb = make([s], [pins], [x], [v])
    cb.step(steps)
    xg, vg = cb.get_state()
    xg = xg.cpu().numpy().reshape(n, n, 3)
    samples = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (1, 2), (n - 2, n // 2), (n // 2, 1),
               (n // 2, n // 2)] + [tuple(int(t) for t in rng.integers(0, n, 2)) for _ in range(40)]
    x64, v64 = x.astype(np.float64), v.astype(np.float64)
    for (r, c) in samples:
        ws, wx, wv, (wr, wc), sh = _window(s, x64, v64, r, c, 2 * steps)
        wp = [p for p in pins if p // n in range(r - 2 * steps, r + 2 * steps + 1)]
        wpins = [(p // n - (r - wr)) * ws["cols"] + (p % n - (c - wc)) for p in wp
                 if 0 <= p // n - (r - wr) < ws["rows"] and 0 <= p % n - (c - wc) < ws["cols"]]
        xr, _ = oracle.step(ws, wx, wv, pins=wpins, steps=steps)
        assert np.abs(xg[r, c] - (xr[wr, wc] + sh)).max() <= X_TOL, (r, c)
    assert cb.status() == 0
    cb.close()


def test_all_nodes_pinned_stay_put():
    s = wl.cloth_spec(9, 13, p=0.5)
    x, v = wl.sag_state(s, np.random.default_rng(92), amp=0.01, vamp=0.1)
    cb = make([s], [list(range(9 * 13))], [x], [v])
    cb.step(25)
    xg, vg = cb.get_state()
    assert torch.equal(xg, pack([x]).cuda()) and float(vg.abs().max()) == 0.0


def test_coincident_nodes_flag_non_finite():
    """Two neighbours at the same position make a zero-length spring: the
    stretch is undefined and the status word reports it."""
    s = wl.cloth_spec(4, 4)
    x, v = wl.noisy_flat_state(s, 0.0, np.random.default_rng(93))
    x[1, 2] = x[1, 1]
    cb = make([s], [[]], [x], [v])
    cb.step(1)
    assert cb.status(clear=True) & 1
