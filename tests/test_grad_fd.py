"""The GPU's hand-written gradients against central finite differences of
the GPU's own FP32 losses (not only through the FP64 oracle).

Eq. 8 (cloth_train_loss): on a 16 x 16 instance of the training workload
(random pins, pressure, scaled stiffness; 8-step unroll; the trainer's
data-scaled initial weights).  The cell behind torch.autograd.Function
(net_forward / net_backward): L = sum(ga * a(w, z)), with the inputs z
perturbed as well.

Directions: one per parameter group (W1, W2, WL, bL, P, WN, WD; for the
cell also the inputs) and 8 over everything.  Each direction d has random
magnitudes |n| (|w| + floor) in the orthant of the gradient's signs, so the
projection g . d has no cancellation and the relative comparison is well
conditioned; a component whose gradient had the wrong sign would enter the
projection with the opposite sign of its true contribution.  The step is
1e-3 of each entry's size (the cell is far from linear over larger steps,
and FP32 rounding of the loss dominates below); the bias enters the output
linearly, so its group takes 1e-1 (for Eq. 8, quadratic in the bias, a step
that moves the loss by 1e-2 of itself).  The perturbed values are FP32, so the
projection uses the perturbation they actually carry, fp32(w + e d) -
fp32(w - e d), not 2 e d.  Tolerance 1e-3 relative.
"""
import numpy as np
import pytest
import torch

from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch
from paper_2403_12820_gb300.net import FP32, N_BLOB, N_PARAMS, CellFunction, Net

pytestmark = pytest.mark.gpu

FD_TOL = 1e-3
GROUPS = [0, 1728, 10944, 11808, 11811, 12835, 12931, N_PARAMS]   # W1 W2 WL bL P WN WD
BIAS = 3                                                         # group index of bL


def directions(n_global=8):
    """(mask over the trainable weights, step) per direction: one per
    group, then n_global over all of them."""
    out = []
    for k, (lo, hi) in enumerate(zip(GROUPS[:-1], GROUPS[1:])):
        m = np.zeros(N_PARAMS)
        m[lo:hi] = 1.0
        out.append((m, 1e-1 if k == BIAS else 1e-3))
    out += [(np.ones(N_PARAMS), 1e-3)] * n_global
    return out


def orthant(rng, g, x, floor):
    return np.sign(g) * (np.abs(x) + floor) * np.abs(rng.normal(size=np.shape(x)))


def test_train_loss_gradient_matches_central_differences():
    from paper_2403_12820_gb300.train import Dataset, Trainer
    data = Dataset(count=4, n=16, steps=24, seed=1004)
    tr = Trainer(data, batch=4, unroll=8, seed=5)
    specs, pins, x0, v0, tg = tr.sample()
    w0 = tr.w.detach().cpu().numpy().astype(np.float32)
    cb = ClothBatch(specs, pins)
    net = Net(w0, FP32)

    def loss(w32, with_grad=False):
        net.set_weights(torch.from_numpy(w32).cuda())
        cb.set_state(x0, v0)
        l, g = cb.train_loss(net, 8, tg, with_grad=with_grad)
        return float(l.item()), (None if g is None else g.cpu().numpy().astype(np.float64))

    L0, g = loss(w0, True)
    assert L0 > 0 and np.all(np.isfinite(g))
    rng = np.random.default_rng(81)
    w64 = w0.astype(np.float64)
    for k, (mask, e) in enumerate(directions()):
        d = np.zeros(N_BLOB)
        d[:N_PARAMS] = mask * orthant(rng, g, w64[:N_PARAMS], 1e-3)
        if k == BIAS:
            # the loss is quadratic in the bias (a is linear in it), so any
            # step is exact; near the optimum its slope is small, so the
            # step is sized to move the loss by 1e-2 of itself, far above
            # the FP32 loss's resolution
            e = 1e-2 * L0 / abs(float(g @ d[:N_PARAMS]))
        wp = (w64 + e * d).astype(np.float32)
        wm = (w64 - e * d).astype(np.float32)
        lp, _ = loss(wp)
        lm, _ = loss(wm)
        proj = float(g @ (wp.astype(np.float64) - wm.astype(np.float64))[:N_PARAMS])
        assert abs((lp - lm) - proj) <= FD_TOL * abs(proj), (k, lp - lm, proj)
    cb.close()
    net.close()


def test_cell_autograd_gradient_matches_central_differences():
    """L = sum(ga * a(w, z)) through CellFunction; the directions also move
    the inputs (one direction over them alone, the global ones over weights
    and inputs together)."""
    rng = np.random.default_rng(82)
    w0 = wl.kaiming_blob(83, in_scale=(50.0,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.1)
    z0 = np.stack([np.concatenate([rng.normal(0, 0.01, (3, 16, 16)), rng.normal(0, 0.1, (3, 16, 16))])
                   for _ in range(2)]).astype(np.float32)
    ga = torch.from_numpy(rng.normal(size=(2, 3, 16, 16)).astype(np.float32)).cuda()
    net = Net(w0, FP32)

    def value(w32, z32):
        with torch.no_grad():
            a = CellFunction.apply(torch.from_numpy(z32).cuda(), torch.from_numpy(w32).cuda(), net)
            return float((a.double() * ga.double()).sum())

    wt = torch.from_numpy(w0).cuda().requires_grad_(True)
    zt = torch.from_numpy(z0).cuda().requires_grad_(True)
    a = CellFunction.apply(zt, wt, net)
    (a * ga).sum().backward()
    gw = wt.grad.cpu().numpy().astype(np.float64)[:N_PARAMS]
    gz = zt.grad.cpu().numpy().astype(np.float64)
    w64, z64 = w0.astype(np.float64), z0.astype(np.float64)
    dirs = [(m, e, 0.0) for (m, e) in directions(n_global=0)]
    dirs += [(np.zeros(N_PARAMS), 1e-3, 1.0)] + [(np.ones(N_PARAMS), 1e-3, 1.0)] * 8
    for k, (mask, e, mz) in enumerate(dirs):
        dw = np.zeros(N_BLOB)
        dw[:N_PARAMS] = mask * orthant(rng, gw, w64[:N_PARAMS], 1e-3)
        dz = mz * orthant(rng, gz, z64, 1e-4)
        wp, wm = (w64 + e * dw).astype(np.float32), (w64 - e * dw).astype(np.float32)
        zp, zm = (z64 + e * dz).astype(np.float32), (z64 - e * dz).astype(np.float32)
        lp, lm = value(wp, zp), value(wm, zm)
        proj = float(gw @ (wp.astype(np.float64) - wm.astype(np.float64))[:N_PARAMS] +
                     (gz * (zp.astype(np.float64) - zm.astype(np.float64))).sum())
        assert abs((lp - lm) - proj) <= FD_TOL * abs(proj), (k, lp - lm, proj)
    net.close()
