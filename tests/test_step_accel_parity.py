"""The network acceleration inside each fused network-step kernel against the
oracle's cell output, element by element.

A network step (Fig. 2, Eq. 5) sets v' = v + dt (a + f_p / m) with a the
cell's output (Eq. 6-7) and f_p the hard-encoded pressure (Eq. 3).  After one
step from (x, v), a_gpu = (v' - v) / dt - f_p(x) / m recovers the kernel's own
a.  Positions after a few steps of 1e-4 s cannot show it (the network moves a
node by about 1e-8 a m per step), so these tests read a directly.  The time
step is 1 s: the FP32 rounding of v' then costs about 6e-8 (|v| / |a| + 1)
relative, far below the tolerance even where a is small (the derivative
branch alone on a 1 x 1 cloth gives |a| near 1e-3 m/s^2 beside |v| near
0.03 m/s).  Only v' is read, so the large step changes nothing else.

Kernels: the tensor-core step (BF16 operands, FP32 accumulation) in its
three tile shapes (14, 10 and 6 output rows), the FP32 CUDA-core step, the
FP32 tensor-core step in its two shapes (10 and 6 rows; each product as three
BF16 products of high and low parts), and the literal-cell step.  Tolerances, normwise per cloth (max
|a_gpu - a_ref| / max |a_ref|): 2e-2 for BF16, 1e-4 for FP32 and the literal
cell.  Besides the whole cell, weight blobs with the linear branch
zeroed (a = N + D) and with only the derivative branch (a = D) keep the
smaller branches from hiding behind the linear one.  Shapes: single nodes,
single rows and columns, exact and ragged tiles of both step kernels, and a
2048 x 2048 cloth sampled on windows of the cell's receptive field.  No pins:
a pinned node's velocity is set, not integrated.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch, pack
from paper_2403_12820_gb300.net import BF16, FP32, Net

pytestmark = pytest.mark.gpu

DT = 1.0
# kind -> (precision, tile choice of tune.net_tile_choices(precision))
NET_KINDS = {"bf16": (BF16, 0), "bf16_r10": (BF16, 1), "bf16_r6": (BF16, 2), "fp32": (FP32, 2), "fp32tc": (FP32, 0),
             "fp32tc_r6": (FP32, 1)}
TOL = {"bf16": 2e-2, "bf16_r10": 2e-2, "bf16_r6": 2e-2, "fp32": 1e-4, "fp32tc": 1e-4, "fp32tc_r6": 1e-4, "pcell": 1e-4}

# blob offsets: W1, W2, WL, bL, P, WN, WD, in_scale, out_scale
O_WL, O_BL, O_P, O_WN, O_WD = 10944, 11808, 11811, 12835, 12931


def normwise(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-30))


def cnn_blob(seed, branches):
    w = wl.kaiming_blob(seed, in_scale=(1 / wl.H_DEFAULT,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3,
                        bias_sigma=0.1)
    if branches in ("ND", "D"):
        w[O_WL:O_P] = 0.0                      # linear branch and its bias
    if branches == "D":
        w[O_WN:O_WD] = 0.0                     # nonlinear branch
    return w


def pcell_weights(seed, branches):
    if branches == "all":
        return wl.pcell_blob(seed)
    rng = np.random.default_rng(seed)          # every branch of one scale
    return np.concatenate([rng.normal(0, 1e4, 36), [0.3, -0.2, -9.81], [625.0]]).astype(np.float32)


def accel_ref(kind, w, spec, x, v):
    if kind == "pcell":
        return oracle.pcell_accel(w.astype(np.float64), spec, x, v)
    return oracle.net_accel(w.astype(np.float64), spec, x, v)


def one_step(kind, w, specs, xs, vs):
    cb = ClothBatch(specs, [[] for _ in specs], dt=DT)
    cb.set_state(pack(xs).cuda(), pack(vs).cuda())
    if kind == "pcell":
        cb.step_pcell(w, 1)
    else:
        prec, choice = NET_KINDS[kind]
        net = Net(w, prec)
        cb.set_net_tile(prec, choice)
        cb.step_net(net, 1)
    _, v1 = cb.get_state()
    got = [t.cpu().numpy().astype(np.float64) for t in cb.split(v1)]
    assert cb.status() == 0
    cb.close()
    return got


def gpu_accel(spec, x, v, v1):
    """a = (v' - v) / dt - f_p(x) / m, in FP64 from the FP32 states."""
    x, v = x.astype(np.float64), v.astype(np.float64)
    return (v1 - v) / DT - oracle.pressure_force(spec, x) / float(spec["m"])


SHAPES = {
    # the step kernels' tiles: R x 26 (tensor cores, R = 14, 10, 6), 14 x 14 (FP32 CUDA cores),
    # 32 x 16 (literal cell)
    "bf16": [(1, 1), (1, 2), (3, 1), (2, 3), (14, 26), (15, 27), (28, 52), (5, 5), (30, 61), (13, 40)],
    "bf16_r10": [(1, 1), (1, 3), (4, 1), (10, 26), (11, 27), (20, 52), (9, 25), (31, 40)],
    "bf16_r6": [(1, 1), (2, 1), (1, 5), (6, 26), (7, 27), (12, 52), (5, 25), (19, 33)],
    "fp32": [(1, 1), (1, 2), (3, 1), (2, 3), (14, 14), (15, 29), (30, 16), (5, 5), (28, 28), (17, 43)],
    "fp32tc": [(1, 1), (1, 2), (3, 1), (2, 3), (10, 26), (11, 27), (20, 52), (5, 5), (31, 61), (13, 40)],
    "fp32tc_r6": [(1, 1), (1, 2), (3, 1), (2, 3), (6, 26), (7, 27), (12, 52), (5, 5), (19, 61), (13, 40)],
    "pcell": [(1, 1), (1, 2), (3, 1), (2, 3), (32, 16), (33, 17), (8, 32), (5, 5), (64, 48), (37, 21)],
}
BRANCHES = {"bf16": ["all", "ND", "D"], "bf16_r10": ["all"], "bf16_r6": ["all"], "fp32": ["all", "ND", "D"],
            "fp32tc": ["all", "ND", "D"], "fp32tc_r6": ["all", "ND", "D"], "pcell": ["all", "mixed"]}
SEED = {"bf16": 301, "bf16_r10": 306, "bf16_r6": 307, "fp32": 302, "fp32tc": 308, "fp32tc_r6": 309, "pcell": 303}


@pytest.mark.parametrize("kind,branches", [(k, b) for k in SHAPES for b in BRANCHES[k]])
def test_step_acceleration_matches_oracle_on_ragged_shapes(kind, branches):
    rng = np.random.default_rng(SEED[kind] + 7 * len(branches))
    specs, xs, vs = [], [], []
    for (r, c) in SHAPES[kind]:
        sp = wl.cloth_spec(r, c, p=rng.normal(0, 0.5), dt=DT)
        x, v = wl.sag_state(sp, rng, amp=0.02, vamp=0.1)
        specs.append(sp); xs.append(x); vs.append(v)
    w = pcell_weights(304, branches) if kind == "pcell" else cnn_blob(305, branches)
    got = one_step(kind, w, specs, xs, vs)
    for b, sp in enumerate(specs):
        a = gpu_accel(sp, xs[b], vs[b], got[b])
        ref = accel_ref(kind, w, sp, xs[b].astype(np.float64), vs[b].astype(np.float64))
        assert np.abs(ref).max() > 0
        err = normwise(a, ref)
        assert err <= TOL[kind], (kind, branches, SHAPES[kind][b], err)


@pytest.mark.parametrize("kind", ["bf16", "fp32", "fp32tc", "pcell"])
def test_step_acceleration_maximum_size_cloth_sampled(kind):
    """One 2048 x 2048 cloth, one step: at sampled nodes (corners, edges,
    random) the kernel's a equals the oracle's cell on the window of the
    receptive field around the node (radius 3 for the two 3x3 trunk
    convolutions and the 3x3 linear branch, 2 for the literal cell's
    stencil; pressure needs 1)."""
    n = 2048
    rad = 2 if kind == "pcell" else 3
    rng = np.random.default_rng({"bf16": 311, "fp32": 312, "fp32tc": 316, "pcell": 313}[kind])
    sp = wl.cloth_spec(n, n, p=0.3, dt=DT)
    x, v = wl.noisy_flat_state(sp, 1e-3, rng)
    v = (v + rng.normal(0, 0.05, v.shape)).astype(np.float32)
    w = pcell_weights(314, "mixed") if kind == "pcell" else cnn_blob(315, "all")
    v1 = one_step(kind, w, [sp], [x], [v])[0].reshape(n, n, 3)
    x64, v64 = x.astype(np.float64), v.astype(np.float64)
    samples = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (1, 1), (2, 1000), (n // 2, n - 2)] + \
              [tuple(int(t) for t in rng.integers(0, n, 2)) for _ in range(30)]
    got, ref = [], []
    for (r, c) in samples:
        r0, r1, c0, c1 = max(0, r - rad), min(n, r + rad + 1), max(0, c - rad), min(n, c + rad + 1)
        ws = dict(sp)
        ws["rows"], ws["cols"] = r1 - r0, c1 - c0
        sh = np.array([c0 * sp["h"], r0 * sp["h"], 0.0])
        xw, vw = x64[r0:r1, c0:c1] - sh, v64[r0:r1, c0:c1]
        a_ref = accel_ref(kind, w, ws, xw, vw)[r - r0, c - c0]
        f_p = oracle.pressure_force(ws, xw)[r - r0, c - c0]
        got.append((v1[r, c] - v64[r, c]) / DT - f_p / float(sp["m"]))
        ref.append(a_ref)
    got, ref = np.array(got), np.array(ref)
    assert normwise(got, ref) <= TOL[kind], normwise(got, ref)
