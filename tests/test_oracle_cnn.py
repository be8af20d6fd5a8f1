"""Pins for the FP64 CNN-cell oracle (Sec. 3.2, Eq. 6-8).

The oracle's direct loops are checked against (a) an independent
formulation built from a library routine (torch.nn.functional.conv2d and
torch.autograd in float64 on the CPU), (b) special weight settings whose
output has a closed form (identity, shifted identity, the 5-point
Laplacian, the tanh and product branches), and (c) central finite
differences of the oracle's own forward for its hand-written backward and
for the unrolled training loss.
"""
import numpy as np
import pytest

import oracle
from paper_2403_12820_gb300 import workloads as wl

torch = pytest.importorskip("torch")
F = torch.nn.functional

C = 32
SL = {
    "W1": slice(0, 1728), "W2": slice(1728, 10944), "WL": slice(10944, 11808), "bL": slice(11808, 11811),
    "P": slice(11811, 12835), "WN": slice(12835, 12931), "WD": slice(12931, 13027),
    "ins": slice(13027, 13033), "outs": slice(13033, 13036),
}


def zero_blob():
    w = np.zeros(oracle.N_BLOB)
    w[SL["ins"]] = 1.0
    w[SL["outs"]] = 1.0
    return w


def torch_cell(w, z):
    """The cell of Eq. 6-7 composed from torch library ops (float64)."""
    w = torch.as_tensor(w)
    W1 = w[SL["W1"]].view(C, 6, 3, 3); W2 = w[SL["W2"]].view(C, C, 3, 3)
    WL = w[SL["WL"]].view(3, C, 3, 3); bL = w[SL["bL"]]
    P = w[SL["P"]].view(C, C, 1, 1); WN = w[SL["WN"]].view(3, C, 1, 1); WD = w[SL["WD"]].view(3, C, 1, 1)
    ins, outs = w[SL["ins"]], w[SL["outs"]]
    zz = z * ins.view(1, 6, 1, 1)
    zu6 = torch.cat([zz[:, :3], torch.zeros_like(zz[:, 3:])], 1)
    zv6 = torch.cat([torch.zeros_like(zz[:, :3]), zz[:, 3:]], 1)
    phi = F.conv2d(F.conv2d(zu6, W1, padding=1), W2, padding=1)
    xi = F.conv2d(F.conv2d(zv6, W1, padding=1), W2, padding=1)
    L = F.conv2d(phi, WL, padding=1) + bL.view(1, 3, 1, 1)
    s = torch.tanh(F.conv2d(phi, P))
    N = F.conv2d(s, WN)
    D = F.conv2d(xi * s, WD)
    return outs.view(1, 3, 1, 1) * (L + N + D)


def rand_blob(seed, scale_in=(3.0, 2.0, 4.0, 0.5, 0.7, 0.3), scale_out=(0.5, 2.0, 1.5)):
    w = wl.kaiming_blob(seed, in_scale=scale_in, out_scale=scale_out, bias_sigma=0.3).astype(np.float64)
    return w


def test_forward_matches_library_conv():
    w = rand_blob(11)
    z = np.random.default_rng(12).normal(size=(2, 6, 9, 13))
    a = oracle.cnn_forward(w, z)
    ref = torch_cell(w, torch.as_tensor(z)).numpy()
    np.testing.assert_allclose(a, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_backward_matches_autograd():
    w = rand_blob(13)
    z = np.random.default_rng(14).normal(size=(2, 6, 7, 10))
    ga = np.random.default_rng(15).normal(size=(2, 3, 7, 10))
    gw, gz = oracle.cnn_backward(w, z, ga)
    wt = torch.tensor(w, requires_grad=True)
    zt = torch.tensor(z, requires_grad=True)
    (torch_cell(wt, zt) * torch.as_tensor(ga)).sum().backward()
    np.testing.assert_allclose(gw, wt.grad.numpy()[:oracle.N_PARAMS], rtol=1e-10, atol=1e-10 * np.abs(gw).max())
    np.testing.assert_allclose(gz, zt.grad.numpy(), rtol=1e-10, atol=1e-10 * np.abs(gz).max())


def _identity_trunk(w, also_v_to_same=False):
    """W1 copies input channel c (and, optionally, c + 3) to trunk channel c;
    W2 copies every trunk channel to itself (centre taps)."""
    W1 = w[SL["W1"]].reshape(C, 6, 3, 3)
    W2 = w[SL["W2"]].reshape(C, C, 3, 3)
    for c in range(3):
        W1[c, c, 1, 1] = 1.0
        W1[c + 3, c + 3, 1, 1] = 1.0
        if also_v_to_same:
            W1[c, c + 3, 1, 1] = 1.0
    for c in range(C):
        W2[c, c, 1, 1] = 1.0


def test_identity_weights_give_scaled_input():
    """Identity trunk, WL = centre tap: a = out_scale (in_scale u + bL)."""
    w = zero_blob()
    _identity_trunk(w)
    WL = w[SL["WL"]].reshape(3, C, 3, 3)
    for c in range(3):
        WL[c, c, 1, 1] = 1.0
    w[SL["bL"]] = [0.1, -0.2, 0.3]
    w[SL["ins"]] = [2, 3, 4, 5, 6, 7]
    w[SL["outs"]] = [0.5, 0.25, 2.0]
    z = np.random.default_rng(16).normal(size=(1, 6, 5, 6))
    a = oracle.cnn_forward(w, z)
    ref = np.array([0.5, 0.25, 2.0]).reshape(1, 3, 1, 1) * (
        np.array([2, 3, 4]).reshape(1, 3, 1, 1) * z[:, :3] + np.array([0.1, -0.2, 0.3]).reshape(1, 3, 1, 1))
    np.testing.assert_allclose(a, ref, rtol=1e-14)


def test_shifted_delta_orientation_and_padding():
    """WL tap (ky, kx) = (0, 2) reads the node one row up and one column to
    the right: L(y, x) = u(y - 1, x + 1), zero outside the grid."""
    w = zero_blob()
    _identity_trunk(w)
    WL = w[SL["WL"]].reshape(3, C, 3, 3)
    for c in range(3):
        WL[c, c, 0, 2] = 1.0
    z = np.random.default_rng(17).normal(size=(1, 6, 6, 7))
    a = oracle.cnn_forward(w, z)
    ref = np.zeros_like(a)
    ref[:, :, 1:, :-1] = z[:, :3, :-1, 1:]
    assert np.array_equal(a, ref)


def test_laplacian_on_linear_branch():
    """WL = 5-point Laplacian stencil per channel gives the discrete
    Laplacian of u with zero Dirichlet padding."""
    w = zero_blob()
    _identity_trunk(w)
    WL = w[SL["WL"]].reshape(3, C, 3, 3)
    for c in range(3):
        WL[c, c] = [[0, 1, 0], [1, -4, 1], [0, 1, 0]]
    z = np.random.default_rng(18).normal(size=(1, 6, 8, 5))
    a = oracle.cnn_forward(w, z)
    u = np.pad(z[:, :3], ((0, 0), (0, 0), (1, 1), (1, 1)))
    lap = u[:, :, :-2, 1:-1] + u[:, :, 2:, 1:-1] + u[:, :, 1:-1, :-2] + u[:, :, 1:-1, 2:] - 4 * u[:, :, 1:-1, 1:-1]
    np.testing.assert_allclose(a, lap, rtol=1e-14, atol=1e-14)


def test_nonlinear_and_derivative_branches_closed_form():
    """Identity trunk mapping u_c and v_c to trunk channel c, P = I:
    N = WN tanh(u), D = WD (v . tanh(u)) per node."""
    w = zero_blob()
    _identity_trunk(w, also_v_to_same=True)
    w[SL["P"]] = np.eye(C).ravel()
    rng = np.random.default_rng(19)
    WN = rng.normal(size=(3, C)); WD = rng.normal(size=(3, C))
    w[SL["WN"]] = WN.ravel(); w[SL["WD"]] = WD.ravel()
    z = rng.normal(size=(1, 6, 4, 5))
    a = oracle.cnn_forward(w, z)
    s = np.tanh(z[0, :3])                   # trunk channels 0..2; the rest are 0
    xi = z[0, 3:]
    ref = np.einsum("oc,cyx->oyx", WN[:, :3], s) + np.einsum("oc,cyx->oyx", WD[:, :3], xi * s)
    np.testing.assert_allclose(a[0], ref, rtol=1e-13, atol=1e-14)


def test_backward_matches_finite_differences():
    w = rand_blob(20)
    rng = np.random.default_rng(21)
    z = rng.normal(size=(1, 6, 6, 5))
    ga = rng.normal(size=(1, 3, 6, 5))
    gw, gz = oracle.cnn_backward(w, z, ga)
    f = lambda ww, zz: float((oracle.cnn_forward(ww, zz) * ga).sum())
    eps = 1e-5
    idx = list(range(SL["bL"].start, SL["bL"].stop))
    for name in ("W1", "W2", "WL", "P", "WN", "WD"):
        s = SL[name]
        idx += list(rng.choice(np.arange(s.start, s.stop), size=6, replace=False))
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += eps; wm[i] -= eps
        num = (f(wp, z) - f(wm, z)) / (2 * eps)
        assert abs(num - gw[i]) <= 1e-7 * max(1.0, abs(num)), (i, num, gw[i])
    for _ in range(6):
        d = rng.normal(size=z.shape)
        num = (f(w, z + eps * d) - f(w, z - eps * d)) / (2 * eps)
        assert abs(num - (gz * d).sum()) <= 1e-7 * max(1.0, abs(num))


# ------------------------------------------------------------------ Eq. 8 loss
def _window(n=10, S=4, seed=22):
    cfg = wl.plain_batch(seed=seed, count=1, side_lo=n, side_hi=n)
    c = cfg["specs"][0]
    pins = cfg["pins"][0]
    x0, v0 = wl.sag_state(c, np.random.default_rng(seed + 1), amp=0.02, vamp=0.05)
    x0 = x0.astype(np.float64); v0 = v0.astype(np.float64)
    xt, vt = oracle.step(c, x0, v0, pins=pins, steps=1)
    targets = [xt]
    for _ in range(S - 1):
        xt, vt = oracle.step(c, xt, vt, pins=pins, steps=1)
        targets.append(xt)
    f = oracle.total_force(c, x0, v0) - oracle.pressure_force(c, x0)
    a_true = f / c["m"]
    h = c["h"]
    w = wl.kaiming_blob(seed + 2, in_scale=(1 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.1)
    return c, pins, x0, v0, np.array(targets), a_true, w.astype(np.float64)


def test_unroll_loss_gradient_matches_finite_differences():
    c, pins, x0, v0, targets, a_true, w = _window()
    loss, gw = oracle.unroll_loss(w, c, pins, x0, v0, targets, a_true, alpha=0.5, g_norm=9.81, h_norm=c["h"])
    assert loss > 0
    f = lambda ww: oracle.unroll_loss(ww, c, pins, x0, v0, targets, a_true, 0.5, 9.81, c["h"], with_grad=False)[0]
    rng = np.random.default_rng(23)
    eps = 1e-4
    idx = list(range(SL["bL"].start, SL["bL"].stop))
    for name in ("W1", "W2", "WL", "P", "WN", "WD"):
        s = SL[name]
        idx += list(rng.choice(np.arange(s.start, s.stop), size=4, replace=False))
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += eps; wm[i] -= eps
        num = (f(wp) - f(wm)) / (2 * eps)
        assert abs(num - gw[i]) <= 1e-6 * max(abs(num), 1e-3 * np.abs(gw).max()), (i, num, gw[i])
    for _ in range(3):
        d = np.zeros_like(w)
        d[:oracle.N_PARAMS] = rng.normal(size=oracle.N_PARAMS)
        d /= np.linalg.norm(d)
        num = (f(w + eps * d) - f(w - eps * d)) / (2 * eps)
        assert abs(num - (gw * d[:oracle.N_PARAMS]).sum()) <= 1e-6 * abs(num)


def test_unroll_loss_zero_for_exact_model():
    """With the data taken from the model's own rollout and a_true set to the
    model's own acceleration, the loss is zero."""
    c, pins, x0, v0, _, _, w = _window(n=8, S=3, seed=30)
    xs, vs = [], []
    x, v = x0, v0
    for _ in range(3):
        x, v = oracle.net_step(w, c, x, v, pins=pins, steps=1)
        xs.append(x)
    a0 = oracle.net_accel(w, c, x0, v0)
    loss, _ = oracle.unroll_loss(w, c, pins, x0, v0, np.array(xs), a0, 0.5, 9.81, c["h"])
    assert loss < 1e-25


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so the update is
    -lr g / (|g| + eps)."""
    rng = np.random.default_rng(24)
    th, g = rng.normal(size=50), rng.normal(size=50)
    th1, m, v = oracle.adam_step(th, g, np.zeros(50), np.zeros(50), t=1, lr=1e-3)
    np.testing.assert_allclose(th1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)
