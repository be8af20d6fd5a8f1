"""Pins of the oracle's moving boundary and friction contact (Sec. 3.1: the
cloth part that "moves along with other objects", and the ball whose friction
prevents relative motion; the framework couples dry friction contact):
Galilean invariance of a step with moving pins, rigid transport of a fully
pinned cloth, and the contact velocity in closed form for the stick case,
frictionless sliding, partial and full Coulomb friction, and separation."""
import numpy as np
import pytest

import oracle
from paper_2403_12820_gb300 import workloads as wl


def _cloth(rows=6, cols=7, drag=0.0, p=0.4, seed=3):
    rng = np.random.default_rng(seed)
    c = wl.cloth_spec(rows, cols, p=p, drag=drag)
    x, v = wl.sag_state(c, rng, amp=0.02, vamp=0.1)
    return c, x.astype(np.float64), v.astype(np.float64)


def test_moving_pins_are_galilean():
    """Without air drag every force depends on relative positions and
    velocities only: pins moving with u from velocities v0 give the fixed-pin
    motion from v0 - u, carried along by t u."""
    c, x0, v0 = _cloth()
    u = np.array([0.3, -0.2, 0.5])
    pins = [0, 6, 20, 41]
    cm = dict(c, pin_v=tuple(u))
    k = 40
    xa, va = oracle.step(cm, x0, v0, pins=pins, steps=k)
    xb, vb = oracle.step(c, x0, v0 - u, pins=pins, steps=k)
    t = k * c["dt"]
    np.testing.assert_allclose(xa, xb + t * u, rtol=0, atol=1e-12)
    np.testing.assert_allclose(va, vb + u, rtol=0, atol=1e-10)
    pm = oracle.pin_mask(c, pins).reshape(6, 7).astype(bool)
    assert np.abs(va[pm] - u).max() == 0.0


def test_fully_pinned_cloth_moves_rigidly():
    c, x0, v0 = _cloth(drag=0.01)
    u = np.array([-0.1, 0.25, 0.05])
    x, v = oracle.step(dict(c, pin_v=tuple(u)), x0, v0, pins=range(42), steps=25)
    np.testing.assert_allclose(x, x0 + 25 * c["dt"] * u, rtol=0, atol=1e-14)
    assert np.array_equal(v, np.broadcast_to(u, v.shape))


def _contact(v, friction, depth=0.01):
    """One node 1 m above a unit sphere's centre along z, moved inside by
    `depth` by the update (acc = 0, dt = 1e-4 s): the outward normal is +z."""
    c = wl.cloth_spec(1, 1, g=(0.0, 0.0, 0.0), drag=0.0)
    c = dict(c, sphere={"center": (0.0, 0.0, -1.0 - 1e-6), "radius": 1.0, "friction": friction})
    v = np.asarray(v, dtype=np.float64).reshape(1, 1, 3)
    x = -c["dt"] * v                                        # lands on the z axis ...
    x[0, 0, 2] -= depth                                     # ... at z = -depth after the update
    x1, v1 = oracle.update(c, x, v, np.zeros((1, 1, 3)))
    assert abs(np.linalg.norm(x1[0, 0] - np.array([0.0, 0.0, -1.0 - 1e-6])) - 1.0) < 1e-12
    return v1[0, 0]


def test_contact_sticks_with_negative_friction():
    assert np.array_equal(_contact([0.3, -0.4, -2.0], -1.0), np.zeros(3))
    assert np.array_equal(_contact([0.3, -0.4, 2.0], -1.0), np.zeros(3))


def test_frictionless_contact_absorbs_only_the_approach():
    np.testing.assert_allclose(_contact([0.3, -0.4, -2.0], 0.0), [0.3, -0.4, 0.0], rtol=0, atol=1e-15)


def test_coulomb_friction_takes_mu_times_the_absorbed_normal_speed():
    vt = np.array([0.3, -0.4])                              # |v_t| = 0.5
    got = _contact([vt[0], vt[1], -1.0], 0.2)               # mu j = 0.2 < 0.5
    np.testing.assert_allclose(got[:2], vt * (0.5 - 0.2) / 0.5, rtol=1e-14, atol=0)
    assert got[2] == 0.0
    assert np.array_equal(_contact([vt[0], vt[1], -1.0], 0.6), np.zeros(3))   # mu j = 0.6 >= 0.5: sticks


def test_separating_node_keeps_its_velocity():
    np.testing.assert_allclose(_contact([0.3, -0.4, 1.5], 0.7), [0.3, -0.4, 1.5], rtol=0, atol=1e-15)


@pytest.mark.parametrize("friction", [-1.0, 0.0, 0.5])
def test_network_step_uses_the_same_constraint(friction):
    """The oracle's network steps take pins and contact from the same update
    as the plain step: with a zero cell they equal the update with the
    pressure acceleration alone."""
    c, x0, v0 = _cloth(rows=8, cols=8)
    c = dict(c, pin_v=(0.0, 0.1, -0.2), sphere={"center": (0.07, 0.07, -0.02), "radius": 0.05,
                                                 "friction": friction})
    w = np.zeros(oracle.PCELL_BLOB)
    w[39] = 1.0
    xs, vs = oracle.pcell_step(w, c, x0, v0, pins=[3, 9], steps=1)
    xr, vr = oracle.update(c, x0, v0, oracle.pressure_force(c, x0) / c["m"], pins=[3, 9])
    assert np.array_equal(xs, xr) and np.array_equal(vs, vr)


def test_unrolled_loss_gradient_with_moving_pins_matches_central_differences():
    """Eq. 8 through a 3-step unroll of the literal cell with pins moving:
    the pinned velocities do not depend on the parameters, so the adjoint
    keeps its form; checked against central differences."""
    s = dict(wl.cloth_spec(5, 6, p=0.4), pin_v=(0.05, -0.02, 0.1))
    rng = np.random.default_rng(17)
    x0, v0 = wl.sag_state(s, rng, amp=0.005, vamp=0.05)
    x0, v0 = x0.astype(np.float64), v0.astype(np.float64)
    pins = [0, 5, 17]
    w = np.asarray(wl.pcell_blob(18), dtype=np.float64)
    tg, xt, vt = [], x0, v0
    for _ in range(3):
        xt, vt = oracle.step(s, xt, vt, pins=pins, steps=1)
        tg.append(xt)
    a_true = (oracle.total_force(s, x0, v0) - oracle.pressure_force(s, x0)) / s["m"]
    args = (s, pins, x0, v0, np.array(tg), a_true, 0.5, 9.81, s["h"])
    loss, gw = oracle.unroll_loss(w, *args, cell="pcell")
    for p in list(range(0, 39, 4)) + [37]:
        eps = 1e-3 * max(1.0, abs(w[p]))
        e = np.zeros(40)
        e[p] = eps
        lp, _ = oracle.unroll_loss(w + e, *args, with_grad=False, cell="pcell")
        lm, _ = oracle.unroll_loss(w - e, *args, with_grad=False, cell="pcell")
        fd = (lp - lm) / (2 * eps)
        # relative 1e-5, plus the rounding of the two losses (~1e-16 |loss|)
        # carried into the difference quotient
        assert abs(gw[p] - fd) <= 1e-5 * abs(fd) + 1e-15 * abs(loss) / eps, (p, gw[p], fd)
    # the recorded targets are the oracle's own moving-pin rollout: pinned
    # nodes sit where the unroll puts them
    pm = oracle.pin_mask(s, pins).reshape(5, 6).astype(bool)
    np.testing.assert_allclose(tg[2][pm], x0[pm] + 3 * s["dt"] * np.asarray(s["pin_v"]), rtol=0, atol=1e-15)
