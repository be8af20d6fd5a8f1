"""Pins for the FP64 mass-spring oracle (Sec. 3.1, Eq. 1-5).

Each test checks the oracle against something it does not compute itself:
closed forms, invariants of the physics, brute force on tiny grids or the
paper's printed spring count.  Together they are chosen so that a dropped
term, a wrong sign, a wrong stencil offset or a swapped operand fails one
of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2403_12820_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def spec(rows, cols, **kw):
    base = dict(h=0.02, m=1e-3, k=(500.0, 250.0, 50.0), mu=0.0, drag=0.0, p=0.0, g=(0.0, 0.0, 0.0), dt=1e-4)
    base.update(kw)
    return wl.cloth_spec(rows, cols, **base)


def noisy(c, sigma, seed, vsig=0.0):
    rng = np.random.default_rng(seed)
    x = wl.rest_grid(c) + rng.normal(0, sigma, size=(c["rows"], c["cols"], 3))
    v = rng.normal(0, vsig, size=x.shape) if vsig else np.zeros_like(x)
    return x, v


# ------------------------------------------------------------------ topology
@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 2), (2, 1), (2, 2), (3, 3), (4, 4), (5, 7), (7, 5), (32, 32), (100, 100)])
def test_spring_counts_closed_form(rows, cols):
    s, sh, b = oracle.spring_counts(rows, cols)
    assert s == rows * (cols - 1) + cols * (rows - 1)
    assert sh == 2 * (rows - 1) * (cols - 1)
    assert b == rows * max(cols - 2, 0) + cols * max(rows - 2, 0)


def test_spring_count_paper_100x100():
    """Sec. 4.1 gives roughly 60 thousand springs for a 100 x 100 grid of mass points."""
    with open(os.path.join(GOLD, "spring_count_100x100.json")) as fh:
        gold = json.load(fh)
    total = sum(oracle.spring_counts(100, 100))
    assert total == gold["closed_form_total"]
    assert abs(total - gold["paper_approx_total"]) / gold["paper_approx_total"] < 0.05


# bit order of the neighbour mask (E, N, W, S, NE, NW, SW, SE, 2E, 2N, 2W, 2S) as (dr, dc)
MASK_OFFSETS = [(0, 1), (1, 0), (0, -1), (-1, 0), (1, 1), (1, -1), (-1, -1), (-1, 1), (0, 2), (2, 0), (0, -2), (-2, 0)]


@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 2), (2, 1), (4, 4), (5, 7), (6, 3)])
def test_neighbor_mask_brute_force(rows, cols):
    """All-pairs classification of node pairs by lattice offset, independent
    of the stencil table: 8 nodes of the 3x3 block plus the 4 nodes two away
    in the cardinal directions (Sec. 3.1)."""
    mask = oracle.neighbor_mask(rows, cols)
    for r in range(rows):
        for c in range(cols):
            expect = set()
            for r2 in range(rows):
                for c2 in range(cols):
                    dr, dc = r2 - r, c2 - c
                    if (dr, dc) == (0, 0):
                        continue
                    near = max(abs(dr), abs(dc)) == 1
                    far = (abs(dr) == 2 and dc == 0) or (dr == 0 and abs(dc) == 2)
                    if near or far:
                        expect.add((dr, dc))
            got = {MASK_OFFSETS[s] for s in range(12) if mask[r, c] >> s & 1}
            assert got == expect, (r, c)


# ------------------------------------------------------------------ forces
@pytest.mark.parametrize("rows,cols", [(1, 2), (3, 3), (5, 7), (16, 16)])
def test_rest_state_zero_force(rows, cols):
    c = spec(rows, cols, mu=0.3)
    X = wl.rest_grid(c)
    f = oracle.internal_force(c, X, np.zeros_like(X))
    assert np.abs(f).max() <= 1e-13 * c["k_struct"] * c["h"]


def test_momentum_conservation():
    c = spec(9, 11, mu=0.05)
    x, v = noisy(c, 2e-3, 1, vsig=0.1)
    f = oracle.internal_force(c, x, v)
    assert np.abs(f).max() > 1e-3
    assert np.abs(f.sum(axis=(0, 1))).max() <= 1e-12 * np.abs(f).sum()


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q if np.linalg.det(q) > 0 else -q


def test_rigid_motion_invariance():
    """f_int(R x + t, R v) = R f_int(x, v): the spring forces are frame independent."""
    c = spec(6, 8, mu=0.07)
    x, v = noisy(c, 3e-3, 2, vsig=0.2)
    R, t = _rot(3), np.array([0.3, -1.2, 2.5])
    f = oracle.internal_force(c, x, v)
    f2 = oracle.internal_force(c, x @ R.T + t, v @ R.T)
    np.testing.assert_allclose(f2, f @ R.T, atol=1e-12 * np.abs(f).max())


def test_mirror_symmetry():
    """Mirroring the cloth about x = w/2 (column c -> cols-1-c) mirrors the forces."""
    c = spec(5, 7, mu=0.05, p=3.0)
    x, v = noisy(c, 2e-3, 4, vsig=0.1)
    w = (c["cols"] - 1) * c["h"]
    xm = x[:, ::-1].copy(); xm[..., 0] = w - xm[..., 0]
    vm = v[:, ::-1].copy(); vm[..., 0] = -vm[..., 0]
    for fn in (lambda X, V: oracle.internal_force(c, X, V),):
        f = fn(x, v)
        fm = fn(xm, vm)
        ref = f[:, ::-1].copy(); ref[..., 0] = -ref[..., 0]
        np.testing.assert_allclose(fm, ref, atol=1e-12 * np.abs(f).max())
    # pressure: the reflection M turns a x b into -M(a x b) while the mirrored
    # lattice swaps each pair's order, so the force is simply mirrored
    fp, fpm = oracle.pressure_force(c, x), oracle.pressure_force(c, xm)
    ref = fp[:, ::-1].copy(); ref[..., 0] = -ref[..., 0]
    np.testing.assert_allclose(fpm, ref, atol=1e-12 * np.abs(fp).max())


@pytest.mark.parametrize("kind", ["struct", "shear", "bend"])
def test_single_spring_hooke(kind):
    """One spring of each type, stretched by e: |f| = k e along the spring,
    pulling the two ends together, equal and opposite (Hooke's law)."""
    e = 3e-4
    if kind == "struct":
        c = spec(1, 2, k=(400.0, 0.0, 0.0)); i, j, Lh, k = (0, 0), (0, 1), 1.0, 400.0
    elif kind == "shear":
        c = spec(2, 2, k=(0.0, 300.0, 0.0)); i, j, Lh, k = (0, 0), (1, 1), math.sqrt(2), 300.0
    else:
        c = spec(1, 3, k=(0.0, 0.0, 70.0)); i, j, Lh, k = (0, 0), (0, 2), 2.0, 70.0
    L = Lh * c["h"]
    X = wl.rest_grid(c)
    d = X[j] - X[i]
    dhat = d / np.linalg.norm(d)
    x = X.copy()
    x[j] = X[i] + dhat * (L + e)           # stretch the spring (i, j) by e
    f = oracle.internal_force(c, x, np.zeros_like(x))
    np.testing.assert_allclose(f[i], k * e * dhat, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(f[j], -k * e * dhat, rtol=1e-9, atol=1e-15)


def test_spring_damping_axial_only():
    """Eq. 2 damps only the relative velocity along the spring."""
    mu = 0.4
    c = spec(1, 2, mu=mu)
    x = wl.rest_grid(c)
    v = np.zeros_like(x); v[0, 1] = [0.5, 0.0, 0.0]
    f = oracle.internal_force(c, x, v)
    np.testing.assert_allclose(f[0, 0], [mu * 0.5, 0, 0], atol=1e-15)   # node 0 dragged along
    np.testing.assert_allclose(f[0, 1], [-mu * 0.5, 0, 0], atol=1e-15)
    v[0, 1] = [0.0, 0.7, -0.2]
    assert np.abs(oracle.internal_force(c, x, v)).max() < 1e-15


def test_external_force_closed_form():
    c = spec(3, 4, drag=0.02, g=(0.1, -0.2, -9.81))
    rng = np.random.default_rng(5)
    v = rng.normal(size=(3, 4, 3))
    f = oracle.external_force(c, v)
    np.testing.assert_allclose(f, c["m"] * np.array(c["g"]) - c["drag"] * v, rtol=1e-15, atol=1e-18)


# ------------------------------------------------------------------ pressure
def test_pressure_flat_lumped_areas():
    """Flat cloth, +z normal: interior p h^2, edge p h^2 / 2, corner p h^2 / 4;
    the total is p w^2 (w = (n-1) h)."""
    n, p = 6, 2.5
    c = spec(n, n, p=p)
    X = wl.rest_grid(c)
    f = oracle.pressure_force(c, X)
    h2 = c["h"] ** 2
    area = np.full((n, n), 1.0)
    area[0, :] = area[-1, :] = area[:, 0] = area[:, -1] = 0.5
    area[0, 0] = area[0, -1] = area[-1, 0] = area[-1, -1] = 0.25
    np.testing.assert_allclose(f[..., 2], p * h2 * area, rtol=1e-12)
    assert np.abs(f[..., :2]).max() < 1e-15
    np.testing.assert_allclose(f.sum(axis=(0, 1)), [0, 0, p * ((n - 1) * c["h"]) ** 2], rtol=1e-12, atol=1e-16)


def test_pressure_total_equals_vector_area():
    """For any deformed state, the summed nodal pressure is p times the
    vector area of the quad mesh, each quad's area being 1/2 (C - A) x (D - B)
    for its corners A=(r,c), B=(r,c+1), C=(r+1,c+1), D=(r+1,c)."""
    c = spec(7, 9, p=-1.7)
    x, _ = noisy(c, 4e-3, 6)
    f = oracle.pressure_force(c, x)
    A, B, Cc, D = x[:-1, :-1], x[:-1, 1:], x[1:, 1:], x[1:, :-1]
    S = 0.5 * np.cross(Cc - A, D - B).sum(axis=(0, 1))
    np.testing.assert_allclose(f.sum(axis=(0, 1)), c["p"] * S, rtol=1e-11, atol=1e-15)


def test_pressure_vjp_matches_finite_differences():
    c = spec(4, 5, p=1.3)
    x, _ = noisy(c, 3e-3, 7)
    rng = np.random.default_rng(8)
    gf = rng.normal(size=x.shape)
    gx = oracle.pressure_vjp(c, x, gf)
    eps = 1e-6
    num = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps; xm[idx] -= eps
        num[idx] = ((oracle.pressure_force(c, xp) - oracle.pressure_force(c, xm)) * gf).sum() / (2 * eps)
    np.testing.assert_allclose(gx, num, rtol=1e-7, atol=1e-12)


# ------------------------------------------------------------------ integration
def test_single_spring_period():
    """1x2 grid, node 0 pinned, g = 0, no damping, axial stretch: the free
    node oscillates with the symplectic-Euler period
    T_d = 2 pi dt / arccos(1 - k dt^2 / (2 m)) (8.8839 ms at k 500, m 1e-3,
    dt 1e-4), within O(dt^2) of 2 pi sqrt(m / k)."""
    k, m, dt = 500.0, 1e-3, 1e-4
    c = spec(1, 2, k=(k, 0.0, 0.0), m=m, dt=dt)
    X = wl.rest_grid(c)
    x = X.copy(); x[0, 1, 0] += 1e-3
    v = np.zeros_like(x)
    # record the free node's displacement for 4000 steps
    traj = []
    for _ in range(4000):
        x, v = oracle.step(c, x, v, pins=[0], steps=1)
        traj.append(x[0, 1, 0] - X[0, 1, 0])
    traj = np.array(traj)
    s = np.sign(traj)
    idx = np.nonzero(s[:-1] != s[1:])[0]
    # linear interpolation of the zero crossings (step index n is time (n+1) dt)
    tc = (idx + 1 + traj[idx] / (traj[idx] - traj[idx + 1])) * dt
    period = 2.0 * np.mean(np.diff(tc))
    Td = 2 * math.pi * dt / math.acos(1 - k * dt * dt / (2 * m))
    assert abs(Td - 8.8839e-3) < 1e-7
    assert abs(period - Td) / Td < 2e-5
    assert abs(period - 2 * math.pi * math.sqrt(m / k)) / Td < 5e-4
    assert np.all(x[0, 0] == X[0, 0])


def test_free_fall_closed_form():
    """Undeformed cloth, no pins, no drag: all springs stay at rest length and
    every node follows v_n = n dt g, z_n = z_0 + g dt^2 n (n + 1) / 2."""
    c = spec(4, 5, g=(0.0, 0.0, -9.81))
    X = wl.rest_grid(c)
    n = 50
    x, v = oracle.step(c, X, np.zeros_like(X), steps=n)
    g, dt = c["g"][2], c["dt"]
    np.testing.assert_allclose(v[..., 2], n * dt * g, rtol=1e-9)
    np.testing.assert_allclose(x[..., 2], g * dt * dt * n * (n + 1) / 2, rtol=1e-9)
    np.testing.assert_allclose(x[..., :2], X[..., :2], atol=1e-15)


def test_drag_closed_form():
    """A lone node under drag only: v_n = v_0 (1 - dt d / m)^n."""
    c = spec(1, 1, drag=0.01, g=(0.0, 0.0, 0.0))
    X = wl.rest_grid(c)
    v0 = np.array([[[0.3, -0.2, 0.5]]])
    n = 200
    x, v = oracle.step(c, X, v0, steps=n)
    fac = (1 - c["dt"] * c["drag"] / c["m"]) ** n
    np.testing.assert_allclose(v, v0 * fac, rtol=1e-12)


def test_pins_hold_position():
    cfg = wl.single_cloth(steps=300)
    c, pins = cfg["specs"][0], cfg["pins"][0]
    x0 = cfg["x"][0].astype(np.float64)
    x, v = oracle.step(c, x0, cfg["v"][0], pins=pins, steps=300)
    flat = x.reshape(-1, 3)
    for p in pins:
        assert np.all(flat[p] == x0.reshape(-1, 3)[p])
        assert np.all(v.reshape(-1, 3)[p] == 0.0)
    assert x[..., 2].min() < -1e-3          # the rest of the cloth falls


def test_sphere_projection():
    """A node found inside the sphere ends on its surface with zero velocity;
    nodes outside are untouched by the contact."""
    R = 0.05
    c = spec(1, 2, k=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0),
             sphere={"center": (0.0, 0.0, -0.0499), "radius": R})
    x = wl.rest_grid(c)
    v = np.zeros_like(x)
    v[0, 0] = [0.0, 0.0, -1.0]         # moves into the sphere this step
    v[0, 1] = [0.0, 0.0, 2.0]          # moves away, stays outside
    x1, v1 = oracle.step(c, x, v, steps=1)
    d = x1[0, 0] - np.array(c["sphere"]["center"])
    assert abs(np.linalg.norm(d) - c["sphere"]["radius"]) < 1e-15
    assert np.all(v1[0, 0] == 0.0)
    np.testing.assert_allclose(x1[0, 1], x[0, 1] + c["dt"] * v[0, 1], rtol=1e-15)
    np.testing.assert_allclose(v1[0, 1], v[0, 1])


def _energy_drift(dt, t_end=0.2, every=0.002):
    c = spec(16, 16, dt=dt, g=(0.0, 0.0, -9.81))
    x, v = noisy(c, 1e-4, 9)
    pins = [15 * 16, 15 * 16 + 15]
    E0 = oracle.energy(c, x, v)
    dev, ke_max = 0.0, 0.0
    k = int(round(every / dt))
    for _ in range(int(round(t_end / every))):
        x, v = oracle.step(c, x, v, pins=pins, steps=k)
        dev = max(dev, abs(oracle.energy(c, x, v) - E0))
        ke_max = max(ke_max, 0.5 * c["m"] * float((v * v).sum()))
    return dev / ke_max


def test_energy_no_secular_drift():
    """Damping, drag and pressure off, two pinned corners: symplectic Euler
    keeps the energy error bounded and first order in dt (halving dt about
    halves it)."""
    d1 = _energy_drift(1e-4)
    d2 = _energy_drift(5e-5)
    assert d1 < 5e-3
    assert 1.6 < d1 / d2 < 2.5, (d1, d2)
