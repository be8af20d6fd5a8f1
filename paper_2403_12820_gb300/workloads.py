"""Seeded synthetic inputs shaped like the paper's cloth scenes.

This module only draws random numbers and fills in parameters; it holds none
of the method's arithmetic.  It serves both the CUDA path and the FP64 oracle
used by the tests: every value is drawn in float64 from a seeded numpy
generator, rounded to float32, and handed to the GPU as float32 and to the
oracle as its exact float64 promotion.

Workloads (sizes follow the paper's 100x100-class square cloths, Sec. 4.1,
and its falling / pinned / pressure / ball scenes, Sec. 3.2.2):
  single_cloth   32x32 cloth, two top corners pinned, Gaussian noise 1e-4 m
  plain_batch    64 cloths, sides U{64..512}, k x U(0.8, 1.2), 1-4 pinned
                 boundary nodes, pressure ~ N(0, 0.5) N/m^2 per cloth
  cnn_batch      32 cloths of 128x128 drawn like plain_batch
  train_set      cloths of 64x64 (random pins, pressure, k scale)
  mixed_batch    16 cloths, sides U{256..1024}, sphere below each cloth
"""
from __future__ import annotations

import numpy as np

N_PARAMS = 13027
N_BLOB = 13036
C = 32

H_DEFAULT = 0.02
M_DEFAULT = 1e-3
K_DEFAULT = (500.0, 250.0, 50.0)
DRAG_DEFAULT = 0.01
G_DEFAULT = (0.0, 0.0, -9.81)
DT_DEFAULT = 1e-4


def f32(v) -> float:
    return float(np.float32(v))


def cloth_spec(rows: int, cols: int, h=H_DEFAULT, m=M_DEFAULT, k=K_DEFAULT, mu=0.0, drag=DRAG_DEFAULT,
               p=0.0, g=G_DEFAULT, dt=DT_DEFAULT, sphere=None, pin_v=None) -> dict:
    """One cloth's parameters, every float rounded to float32.  sphere:
    {center, radius[, friction]}; pin_v: the velocity the pinned nodes move
    with (absent: they stay in place)."""
    spec = {
        "rows": int(rows), "cols": int(cols), "h": f32(h), "m": f32(m),
        "k_struct": f32(k[0]), "k_shear": f32(k[1]), "k_bend": f32(k[2]),
        "mu": f32(mu), "drag": f32(drag), "p": f32(p), "g": [f32(a) for a in g], "dt": f32(dt),
    }
    if sphere is not None:
        spec["sphere"] = {"center": [f32(a) for a in sphere["center"]], "radius": f32(sphere["radius"])}
        if "friction" in sphere:
            spec["sphere"]["friction"] = f32(sphere["friction"])
    if pin_v is not None:
        spec["pin_v"] = [f32(a) for a in pin_v]
    return spec


def rest_grid(spec: dict) -> np.ndarray:
    """Undeformed lattice positions (c h, r h, 0), float64 of float32 values."""
    rows, cols, h = spec["rows"], spec["cols"], spec["h"]
    X = np.zeros((rows, cols, 3))
    X[..., 0] = np.arange(cols)[None, :] * h
    X[..., 1] = np.arange(rows)[:, None] * h
    return X


def noisy_flat_state(spec: dict, sigma: float, rng: np.random.Generator):
    """Flat cloth in the xy-plane plus N(0, sigma^2) noise on every coordinate;
    zero velocity.  Returns float32 arrays (rows, cols, 3)."""
    x = rest_grid(spec) + rng.normal(0.0, sigma, size=(spec["rows"], spec["cols"], 3))
    return x.astype(np.float32), np.zeros_like(x, dtype=np.float32)


def boundary_nodes(rows: int, cols: int) -> np.ndarray:
    idx = [r * cols + c for r in range(rows) for c in range(cols)
           if r == 0 or r == rows - 1 or c == 0 or c == cols - 1]
    return np.array(idx, dtype=np.int64)


# --------------------------------------------------------------- workloads
def single_cloth(seed: int = 1001, n: int = 32, steps: int = 2000) -> dict:
    """32x32, h 0.02 m, 1e-3 kg/node, k 500/250/50 N/m, drag 0.01, gravity
    -9.81 z, corners (n-1, 0) and (n-1, n-1) pinned, dt 1e-4 s, noise 1e-4 m."""
    rng = np.random.default_rng(seed)
    spec = cloth_spec(n, n)
    x, v = noisy_flat_state(spec, 1e-4, rng)
    pins = [(n - 1) * n + 0, (n - 1) * n + (n - 1)]
    return {"specs": [spec], "pins": [pins], "x": [x], "v": [v], "steps": steps}


def plain_batch(seed: int = 1002, count: int = 64, side_lo: int = 64, side_hi: int = 512,
                steps: int = 10000) -> dict:
    """Batch of square cloths with uneven sides, scaled stiffness, 1-4 pinned
    boundary nodes and a per-cloth pressure ("wind") ~ N(0, 0.5) N/m^2."""
    rng = np.random.default_rng(seed)
    specs, pins, xs, vs = [], [], [], []
    sides = rng.integers(side_lo, side_hi + 1, size=count)
    for b in range(count):
        n = int(sides[b])
        ks = rng.uniform(0.8, 1.2)
        p = rng.normal(0.0, 0.5)
        spec = cloth_spec(n, n, k=tuple(kk * ks for kk in K_DEFAULT), p=p)
        npin = int(rng.integers(1, 5))
        bnd = boundary_nodes(n, n)
        pin = sorted(int(i) for i in rng.choice(bnd, size=npin, replace=False))
        x, v = noisy_flat_state(spec, 1e-4, rng)
        specs.append(spec); pins.append(pin); xs.append(x); vs.append(v)
    return {"specs": specs, "pins": pins, "x": xs, "v": vs, "steps": steps}


def sag_state(spec: dict, rng: np.random.Generator, amp: float = 0.05, vamp: float = 0.2,
              sigma: float = 1e-4):
    """A deformed, moving cloth: a smooth random sag (a few low Fourier modes,
    largest displacement about `amp` x cloth width) plus noise, and a smooth
    random velocity field of size about `vamp` m/s.  float32 (rows, cols, 3)."""
    rows, cols, h = spec["rows"], spec["cols"], spec["h"]
    w = max(rows, cols) * h
    yy, xx = np.meshgrid(np.linspace(0, 1, rows), np.linspace(0, 1, cols), indexing="ij")
    u = np.zeros((rows, cols, 3))
    v = np.zeros((rows, cols, 3))
    for _ in range(3):
        kx, ky = rng.integers(1, 4, size=2)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        mode = np.sin(np.pi * kx * xx + ph[0]) * np.sin(np.pi * ky * yy + ph[1])
        u += (amp * w / 3.0) * mode[..., None] * rng.normal(0.0, [0.2, 0.2, 1.0])
        v += (vamp / 3.0) * mode[..., None] * rng.normal(0.0, [0.3, 0.3, 1.0])
    u += rng.normal(0.0, sigma, size=u.shape)
    x = rest_grid(spec) + u
    return x.astype(np.float32), v.astype(np.float32)


def cnn_batch(seed: int = 1003, count: int = 32, n: int = 128, steps: int = 1000) -> dict:
    """Batch of 128x128 cloths drawn like the plain batch (flat + 1e-4 m
    noise, 1-4 pinned boundary nodes, pressure ~ N(0, 0.5), stiffness x
    U(0.8, 1.2)), so that after a few plain steps their states look like the
    training trajectories; the network workload starts from the state after
    100 plain steps (the caller steps them)."""
    return plain_batch(seed=seed, count=count, side_lo=n, side_hi=n, steps=steps)


def mixed_batch(seed: int = 1005, count: int = 16, side_lo: int = 256, side_hi: int = 1024,
                steps: int = 5000) -> dict:
    """Large cloths over a sphere of radius 0.3 w centred under the cloth
    middle at depth R + 0.05 w; no pins; pressure ~ N(0, 0.5)."""
    rng = np.random.default_rng(seed)
    specs, pins, xs, vs = [], [], [], []
    sides = rng.integers(side_lo, side_hi + 1, size=count)
    for b in range(count):
        n = int(sides[b])
        w = (n - 1) * H_DEFAULT
        R = 0.3 * w
        sph = {"center": (w / 2, w / 2, -R - 0.05 * w), "radius": R}
        spec = cloth_spec(n, n, p=rng.normal(0.0, 0.5), sphere=sph)
        x, v = noisy_flat_state(spec, 1e-4, rng)
        specs.append(spec); pins.append([]); xs.append(x); vs.append(v)
    return {"specs": specs, "pins": pins, "x": xs, "v": vs, "steps": steps}


def train_cloths(seed: int = 1004, count: int = 512, n: int = 64) -> dict:
    """Initial states for training trajectories: random 1-4 pinned boundary
    nodes, pressure ~ N(0, 0.5), stiffness x U(0.8, 1.2)."""
    return plain_batch(seed=seed, count=count, side_lo=n, side_hi=n, steps=200)


# --------------------------------------------------------------- weights
def kaiming_blob(seed: int = 2003, in_scale=(1.0,) * 6, out_scale=(1.0,) * 3, bias_sigma: float = 0.0) -> np.ndarray:
    """Weight blob of the CNN cell: W1[32][6][3][3], W2[32][32][3][3],
    WL[3][32][3][3], bL[3], P[32][32], WN[3][32], WD[3][32], in_scale[6],
    out_scale[3].  Weights ~ N(0, 2 / fan_in) (He et al. 2015), fan_in =
    Cin * kh * kw; bias N(0, bias_sigma^2).  float32."""
    rng = np.random.default_rng(seed)
    parts = [
        rng.normal(0.0, np.sqrt(2.0 / 54), size=C * 6 * 9),
        rng.normal(0.0, np.sqrt(2.0 / 288), size=C * C * 9),
        rng.normal(0.0, np.sqrt(2.0 / 288), size=3 * C * 9),
        rng.normal(0.0, bias_sigma, size=3) if bias_sigma > 0 else np.zeros(3),
        rng.normal(0.0, np.sqrt(2.0 / 32), size=C * C),
        rng.normal(0.0, np.sqrt(2.0 / 32), size=3 * C),
        rng.normal(0.0, np.sqrt(2.0 / 32), size=3 * C),
        np.asarray(in_scale, dtype=np.float64),
        np.asarray(out_scale, dtype=np.float64),
    ]
    blob = np.concatenate(parts).astype(np.float32)
    assert blob.shape == (N_BLOB,)
    return blob


def pcell_blob(seed: int = 2005, h: float = H_DEFAULT, m: float = M_DEFAULT, k=K_DEFAULT,
               g=G_DEFAULT) -> np.ndarray:
    """Weights of the literal cell (40 floats: w_L[12], w_N[12], w_D[12],
    b_L[3], alpha), spring-like: w_L = k_type / m scattered by U(0.9, 1.1)
    per channel, nonlinear and derivative weights of a tenth of that scale
    with random signs, b_L = g, alpha = 1 / (2 h)^2 so the ISRU bends at
    displacements of the lattice scale; rounded to float32."""
    rng = np.random.default_rng(seed)
    kc = np.array([k[0]] * 4 + [k[1]] * 4 + [k[2]] * 4) / m
    w = np.zeros(40)
    w[0:12] = kc * rng.uniform(0.9, 1.1, 12)
    w[12:24] = 0.1 * kc * h * rng.choice([-1.0, 1.0], 12) * rng.uniform(0.5, 1.5, 12)
    w[24:36] = 0.1 * kc * rng.choice([-1.0, 1.0], 12) * rng.uniform(0.5, 1.5, 12) * 1e-3
    w[36:39] = g
    w[39] = 1.0 / (2.0 * h) ** 2
    return w.astype(np.float32)


def de_draws(seed: int = 2007, pop: int = 36, dim: int = 6, generations: int = 20) -> dict:
    """Random numbers of one differential-evolution run, drawn up front:
    init (pop, dim) uniforms in [0, 1) for the starting population; idx
    (generations, pop, 3) three distinct members other than i for member i;
    jrand (generations, pop) a component index; cross (generations, pop,
    dim) uniforms in [0, 1) for the crossover."""
    if pop < 4 or dim < 1 or generations < 0:
        raise ValueError("differential evolution needs pop >= 4, dim >= 1, generations >= 0")
    rng = np.random.default_rng(seed)
    init = rng.random((pop, dim))
    idx = np.empty((generations, pop, 3), dtype=np.int64)
    for g in range(generations):
        for i in range(pop):
            k = rng.choice(pop - 1, size=3, replace=False)
            idx[g, i] = k + (k >= i)
    jrand = rng.integers(0, dim, size=(generations, pop))
    cross = rng.random((generations, pop, dim))
    return {"init": init, "idx": idx, "jrand": jrand, "cross": cross}
