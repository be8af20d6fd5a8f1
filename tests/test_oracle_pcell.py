"""Pins of the oracle's literal cell (Eq. 6-7 with frozen difference
channels and ISRU, Fig. 1) against what the mathematics fixes, each by a
route that does not reuse the oracle's channel table:

- zero-rest-length springs: with w_L = k_type / m, w_N = w_D = 0 and
  b_L = g the cell is Hooke's law for springs of zero rest length over the
  stencil, checked against an all-pairs loop that classifies node pairs by
  their lattice offset;
- two nodes: all three branches written out by hand;
- ISRU saturation: sigma(z) -> 1 / sqrt(alpha) for large z;
- invariances: a rigid translation of x, a uniform velocity;
- mirror symmetry: reversing the columns with mirrored weights mirrors a;
- the step: with zero weights and b_L = g, symplectic-Euler free fall.
"""
import numpy as np
import pytest

import oracle
from paper_2403_12820_gb300 import workloads as wl


def rand_state(s, seed, amp=0.01, vamp=0.2):
    rng = np.random.default_rng(seed)
    x = oracle.rest_positions(s) + rng.normal(0, amp, (s["rows"], s["cols"], 3))
    v = rng.normal(0, vamp, (s["rows"], s["cols"], 3))
    return x, v


def rand_w(seed, alpha=1.0):
    rng = np.random.default_rng(seed)
    w = rng.normal(0, 1, 40)
    w[39] = alpha
    return w


@pytest.mark.parametrize("shape", [(1, 1), (1, 2), (3, 4), (6, 5)])
def test_zero_rest_length_springs_all_pairs(shape):
    rows, cols = shape
    s = wl.cloth_spec(rows, cols)
    x, v = rand_state(s, 1)
    ks, ksh, kb, m = s["k_struct"], s["k_shear"], s["k_bend"], s["m"]
    w = np.zeros(40)
    # channels: 4 structural, 4 shear, 4 bending (E W N S NE NW SE SW E2 W2 N2 S2)
    w[0:4] = ks / m
    w[4:8] = ksh / m
    w[8:12] = kb / m
    w[36:39] = s["g"]
    w[39] = 1.0
    a = oracle.pcell_accel(w, s, x, v)
    ref = np.zeros_like(x)
    for i in range(rows * cols):
        ri, ci = divmod(i, cols)
        ref[ri, ci] = s["g"]
        for j in range(rows * cols):
            rj, cj = divmod(j, cols)
            dr, dc = abs(rj - ri), abs(cj - ci)
            if (dr, dc) in ((0, 1), (1, 0)):
                k = ks
            elif (dr, dc) == (1, 1):
                k = ksh
            elif (dr, dc) in ((0, 2), (2, 0)):
                k = kb
            else:
                continue
            ref[ri, ci] += k / m * (x[rj, cj] - x[ri, ci])
    assert np.abs(a - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1.0)


def test_two_nodes_by_hand():
    s = wl.cloth_spec(1, 2)
    x, v = rand_state(s, 2)
    w = rand_w(3, alpha=2.5)
    a = oracle.pcell_accel(w, s, x, v)
    isru = lambda z: z / np.sqrt(1 + 2.5 * z * z)  # noqa: E731
    d = x[0, 1] - x[0, 0]
    e = v[0, 1] - v[0, 0]
    # node 0 sees its E neighbour (channel 0), node 1 its W neighbour (channel 1)
    ref0 = w[0] * d + w[12] * isru(d) + w[24] * e * isru(d) + w[36:39]
    ref1 = w[1] * (-d) + w[13] * isru(-d) + w[25] * (-e) * isru(-d) + w[36:39]
    assert np.allclose(a[0, 0], ref0, rtol=1e-14, atol=1e-14)
    assert np.allclose(a[0, 1], ref1, rtol=1e-14, atol=1e-14)


def test_isru_saturation():
    s = wl.cloth_spec(1, 2)
    x = oracle.rest_positions(s)
    x[0, 1] += np.array([1e6, -1e6, 0.0])
    w = np.zeros(40)
    w[12] = 1.0          # nonlinear branch of channel E only
    w[39] = 4.0
    a = oracle.pcell_accel(w, s, x, np.zeros_like(x))
    assert np.allclose(a[0, 0], [0.5, -0.5, 0.0], atol=1e-9)
    assert np.allclose(a[0, 1], 0.0)


def test_translation_and_uniform_velocity_invariance():
    s = wl.cloth_spec(5, 7)
    x, v = rand_state(s, 4)
    w = rand_w(5)
    a = oracle.pcell_accel(w, s, x, v)
    a_t = oracle.pcell_accel(w, s, x + np.array([0.3, -1.2, 2.0]), v + np.array([1.5, 0.2, -3.0]))
    assert np.abs(a - a_t).max() <= 1e-12
    w_d = np.zeros(40)
    w_d[24:36] = 1.0
    w_d[39] = 1.0
    assert np.abs(oracle.pcell_accel(w_d, s, x, np.ones_like(v) * 0.7)).max() <= 1e-15


@pytest.mark.parametrize("branch", ["LN", "D"])
def test_mirror_symmetry(branch):
    """Reversing the columns (x -> w - x) with E <-> W, NE <-> NW, SE <-> SW,
    E2 <-> W2 swapped in every branch mirrors the field.  The linear and
    nonlinear branches are odd in the difference, so their x component
    changes sign; the derivative branch multiplies two x differences per
    coordinate and its x component keeps its sign."""
    s = wl.cloth_spec(4, 6)
    x, v = rand_state(s, 6)
    w = rand_w(7)
    if branch == "LN":
        w[24:36] = 0.0
    else:
        w[0:24] = 0.0
        w[36:39] = 0.0
    width = (s["cols"] - 1) * s["h"]
    flip = np.array([-1.0, 1.0, 1.0])
    xm = x[:, ::-1].copy() * flip
    xm[..., 0] += width
    vm = v[:, ::-1].copy() * flip
    perm = [1, 0, 2, 3, 5, 4, 7, 6, 9, 8, 10, 11]
    wm = w.copy()
    for b in range(3):
        wm[12 * b:12 * b + 12] = w[12 * b:12 * b + 12][perm]
    wm[36] = -w[36]
    a = oracle.pcell_accel(w, s, x, v)
    am = oracle.pcell_accel(wm, s, xm, vm)
    sign = flip if branch == "LN" else np.ones(3)
    assert np.abs(am[:, ::-1] * sign - a).max() <= 1e-12


def test_step_free_fall_closed_form():
    s = wl.cloth_spec(3, 4)
    x0, v0 = rand_state(s, 8, amp=0.0)
    w = np.zeros(40)
    w[36:39] = s["g"]
    w[39] = 1.0
    n = 25
    x, v = oracle.pcell_step(w, s, x0, v0, steps=n)
    g = np.asarray(s["g"])
    dt = s["dt"]
    # symplectic Euler: v_n = v0 + n dt g, x_n = x0 + n dt v0 + dt^2 g n (n+1) / 2
    assert np.allclose(v, v0 + n * dt * g, rtol=0, atol=1e-13)
    assert np.allclose(x, x0 + n * dt * v0 + dt * dt * g * n * (n + 1) / 2, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- backward
def test_backward_matches_central_differences():
    """Gradient of sum(ga . a) for every trainable parameter and for random
    directions in x and v, against central differences (eps 1e-6)."""
    s = wl.cloth_spec(4, 5)
    x, v = rand_state(s, 9)
    w = rand_w(10, alpha=300.0)
    ga = np.random.default_rng(11).normal(size=x.shape)
    f = lambda ww, xx, vv: float((ga * oracle.pcell_accel(ww, s, xx, vv)).sum())  # noqa: E731
    gw, gx, gv = oracle.pcell_backward(w, s, x, v, ga)
    eps = 1e-6
    for p in range(39):
        e = np.zeros(40)
        e[p] = eps
        fd = (f(w + e, x, v) - f(w - e, x, v)) / (2 * eps)
        assert abs(gw[p] - fd) <= 1e-6 * max(1.0, abs(fd)), p
    assert gw[39] == 0.0
    rng = np.random.default_rng(12)
    for _ in range(4):
        dx, dv = rng.normal(size=x.shape) * 1e-3, rng.normal(size=v.shape)
        dx /= np.linalg.norm(dx); dv /= np.linalg.norm(dv)
        fdx = (f(w, x + eps * dx, v) - f(w, x - eps * dx, v)) / (2 * eps)
        fdv = (f(w, x, v + eps * dv) - f(w, x, v - eps * dv)) / (2 * eps)
        assert abs((gx * dx).sum() - fdx) <= 1e-6 * max(1.0, abs(fdx))
        assert abs((gv * dv).sum() - fdv) <= 1e-6 * max(1.0, abs(fdv))


def test_backward_matches_torch_autograd():
    """The cell rewritten as torch ops on CPU (FP64, shifted slices per
    channel), differentiated by autograd: a second reference."""
    torch = pytest.importorskip("torch")
    s = wl.cloth_spec(5, 6)
    x, v = rand_state(s, 13)
    w = rand_w(14, alpha=50.0)
    ga = np.random.default_rng(15).normal(size=x.shape)
    X = torch.tensor(x, requires_grad=True)
    V = torch.tensor(v, requires_grad=True)
    Wt = torch.tensor(w, requires_grad=True)
    rows, cols = s["rows"], s["cols"]
    a = Wt[36:39].expand(rows, cols, 3).clone()
    for ch, (dy, dx) in enumerate(oracle.PCELL_CHANNELS):
        ys, xs_ = slice(max(0, -dy), rows - max(0, dy)), slice(max(0, -dx), cols - max(0, dx))
        yj, xj = slice(max(0, dy), rows - max(0, -dy)), slice(max(0, dx), cols - max(0, -dx))
        phi = X[yj, xj] - X[ys, xs_]
        xi = V[yj, xj] - V[ys, xs_]
        sg = phi / torch.sqrt(1 + Wt[39] * phi * phi)
        term = torch.zeros(rows, cols, 3, dtype=torch.float64)
        term[ys, xs_] = Wt[ch] * phi + Wt[12 + ch] * sg + Wt[24 + ch] * xi * sg
        a = a + term
    assert np.abs(a.detach().numpy() - oracle.pcell_accel(w, s, x, v)).max() <= 1e-12
    (a * torch.tensor(ga)).sum().backward()
    gw, gx, gv = oracle.pcell_backward(w, s, x, v, ga)
    assert np.abs(gw[:39] - Wt.grad.numpy()[:39]).max() <= 1e-9 * np.abs(gw).max()
    assert np.abs(gx - X.grad.numpy()).max() <= 1e-9 * np.abs(gx).max()
    assert np.abs(gv - V.grad.numpy()).max() <= 1e-9 * np.abs(gv).max()


def test_unrolled_loss_gradient_matches_central_differences():
    """Eq. 8 through a 3-step unroll with the literal cell: the adjoint's
    parameter gradient against central differences of the loss."""
    s = wl.cloth_spec(5, 6, p=0.4)
    x0, v0 = rand_state(s, 17, amp=0.005, vamp=0.05)
    pins = [0, 5]
    w = np.asarray(wl.pcell_blob(18), dtype=np.float64)
    tg, xt, vt = [], x0, v0
    for _ in range(3):
        xt, vt = oracle.step(s, xt, vt, pins=pins, steps=1)
        tg.append(xt)
    a_true = (oracle.total_force(s, x0, v0) - oracle.pressure_force(s, x0)) / s["m"]
    args = (s, pins, x0, v0, np.array(tg), a_true, 0.5, 9.81, s["h"])
    loss, gw = oracle.unroll_loss(w, *args, cell="pcell")
    for p in list(range(0, 39, 3)) + [36, 37, 38]:
        eps = 1e-3 * max(1.0, abs(w[p]))   # the loss is ~1e6: a smaller step drowns in rounding
        e = np.zeros(40)
        e[p] = eps
        lp, _ = oracle.unroll_loss(w + e, *args, with_grad=False, cell="pcell")
        lm, _ = oracle.unroll_loss(w - e, *args, with_grad=False, cell="pcell")
        fd = (lp - lm) / (2 * eps)
        assert abs(gw[p] - fd) <= 1e-5 * max(abs(fd), 1e-12 * abs(loss) / eps), (p, gw[p], fd)
