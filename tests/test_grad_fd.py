"""The GPU's hand-written gradients against central finite differences of
the GPU's own FP32 losses (not only through the FP64 oracle).

Eq. 8 (cloth_train_loss): on a 16 x 16 instance of the training workload
(random pins, pressure, scaled stiffness; 8-step unroll; the trainer's
data-scaled initial weights), the loss difference along 8 random directions
over the trainable weights against the gradient's projection.
The cell behind torch.autograd.Function (net_forward / net_backward): the
same along 8 random directions over the weights and the inputs together.

Each direction's step is sized so the loss moves by about 1e-3 of its size
(for the cell's signed sum, 1e-4 of the sum of the terms' magnitudes): the
FP32 loss's rounding noise (about 1e-7 relative) then costs about 1e-4 of the
difference, and the third-order terms the central difference leaves are
below that.
The perturbed weights are FP32, so the projection uses the perturbation they
actually carry (fp32(w + e d) - w), not e d.  Tolerance 1e-3 relative.
"""
import numpy as np
import pytest
import torch

from paper_2403_12820_gb300 import workloads as wl
from paper_2403_12820_gb300.cloth import ClothBatch
from paper_2403_12820_gb300.net import FP32, N_BLOB, N_PARAMS, CellFunction, Net

pytestmark = pytest.mark.gpu

FD_TOL = 1e-3


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
    for k in range(8):
        d = np.zeros(N_BLOB)
        d[:N_PARAMS] = rng.normal(size=N_PARAMS) * (np.abs(w64[:N_PARAMS]) + 1e-3)
        gd = float(g @ d[:N_PARAMS])
        eps = 1e-3 * L0 / abs(gd)
        wp = (w64 + eps * d).astype(np.float32)
        wm = (w64 - eps * d).astype(np.float32)
        lp, _ = loss(wp)
        lm, _ = loss(wm)
        proj = float(g @ (wp.astype(np.float64) - wm.astype(np.float64))[:N_PARAMS])
        assert abs((lp - lm) - proj) <= FD_TOL * abs(proj), (k, lp - lm, proj)
    cb.close()
    net.close()


def test_cell_autograd_gradient_matches_central_differences():
    """L = sum(ga * a(w, z)) through CellFunction; directions over the
    weights and the inputs together."""
    rng = np.random.default_rng(82)
    w0 = wl.kaiming_blob(83, in_scale=(50.0,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.1)
    z0 = np.stack([np.concatenate([rng.normal(0, 0.01, (3, 16, 16)), rng.normal(0, 0.1, (3, 16, 16))])
                   for _ in range(2)]).astype(np.float32)
    ga = torch.from_numpy(rng.normal(size=(2, 3, 16, 16)).astype(np.float32)).cuda()
    net = Net(w0, FP32)

    def value(w32, z32):
        with torch.no_grad():
            a = CellFunction.apply(torch.from_numpy(z32).cuda(), torch.from_numpy(w32).cuda(), net)
            return float((a.double() * ga.double()).sum()), float((a.double() * ga.double()).abs().sum())

    wt = torch.from_numpy(w0).cuda().requires_grad_(True)
    zt = torch.from_numpy(z0).cuda().requires_grad_(True)
    a = CellFunction.apply(zt, wt, net)
    (a * ga).sum().backward()
    gw = wt.grad.cpu().numpy().astype(np.float64)[:N_PARAMS]
    gz = zt.grad.cpu().numpy().astype(np.float64)
    _, mag = value(w0, z0)
    w64, z64 = w0.astype(np.float64), z0.astype(np.float64)
    for k in range(8):
        dw = np.zeros(N_BLOB)
        dw[:N_PARAMS] = rng.normal(size=N_PARAMS) * (np.abs(w64[:N_PARAMS]) + 1e-3)
        dz = rng.normal(size=z0.shape) * (np.abs(z64) + 1e-4)
        gd = float(gw @ dw[:N_PARAMS] + (gz * dz).sum())
        eps = 1e-4 * mag / abs(gd)
        wp, wm = (w64 + eps * dw).astype(np.float32), (w64 - eps * dw).astype(np.float32)
        zp, zm = (z64 + eps * dz).astype(np.float32), (z64 - eps * dz).astype(np.float32)
        lp, _ = value(wp, zp)
        lm, _ = value(wm, zm)
        proj = float(gw @ (wp.astype(np.float64) - wm.astype(np.float64))[:N_PARAMS] +
                     (gz * (zp.astype(np.float64) - zm.astype(np.float64))).sum())
        assert abs((lp - lm) - proj) <= FD_TOL * abs(proj), (k, lp - lm, proj)
    net.close()
