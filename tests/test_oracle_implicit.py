"""Pins of the oracle's implicit (linearised backward Euler) plain step: the
closed-form backward Euler step of one axial spring with drag, the spring
Jacobian against central differences of the Eq. 1 force, its symmetry and
translation invariance, momentum conservation of a free cloth, and the
step's agreement with the explicit step to third order in the time step."""
import numpy as np

import oracle
from paper_2403_12820_gb300 import workloads as wl


def _cloth(rows=5, cols=6, p=0.0, drag=0.0, g=(0.0, 0.0, 0.0), seed=2, scale=1.0):
    rng = np.random.default_rng(seed)
    c = wl.cloth_spec(rows, cols, p=p, drag=drag, g=g)
    x, v = wl.sag_state(c, rng, amp=0.01, vamp=0.05)
    x = x.astype(np.float64) * scale
    return c, x, v.astype(np.float64)


def test_single_axial_spring_is_backward_euler_in_closed_form():
    k, m, d, h, L = 500.0, 1e-3, 0.01, 1e-3, 0.02
    c = wl.cloth_spec(1, 2, k=(k, 0.0, 0.0), drag=d, g=(0.0, 0.0, 0.0), dt=h, h=L, m=m)
    h, m, k, L, d = c["dt"], c["m"], c["k_struct"], c["h"], c["drag"]   # the float32-rounded values
    e, w = 0.003, -0.7
    x = np.array([[[0.0, 0.0, 0.0], [L + e, 0.0, 0.0]]])
    v = np.array([[[0.0, 0.0, 0.0], [w, 0.0, 0.0]]])
    x1, v1 = oracle.implicit_step(c, x, v, pins=[0])
    want_v = (m * w - h * k * e) / (m + h * d + h * h * k)
    np.testing.assert_allclose(v1[0, 1], [want_v, 0.0, 0.0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(x1[0, 1], [L + e + h * want_v, 0.0, 0.0], rtol=1e-12, atol=1e-15)
    assert np.array_equal(x1[0, 0], x[0, 0]) and np.array_equal(v1[0, 0], v[0, 0])
    # backward Euler loses energy on the undamped spring
    cu = dict(c, drag=0.0)
    x2, v2 = oracle.implicit_step(cu, x, v, pins=[0])
    energy = lambda xx, vv: 0.5 * m * vv[0, 1, 0] ** 2 + 0.5 * k * (xx[0, 1, 0] - L) ** 2
    assert energy(x2, v2) < energy(x, v)


def test_jacobian_matches_central_differences_of_the_spring_force():
    """On a stretched cloth (every spring longer than its rest length, so the
    clamp is inactive) K is the exact derivative of Eq. 1."""
    c, x, v = _cloth(scale=1.03)
    K = oracle.stiffness(c, x).toarray()
    n = x.size
    rng = np.random.default_rng(3)
    for _ in range(6):
        dirn = rng.normal(size=n)
        eps = 1e-7
        fp = oracle.internal_force(c, x + eps * dirn.reshape(x.shape), v).reshape(-1)
        fm = oracle.internal_force(c, x - eps * dirn.reshape(x.shape), v).reshape(-1)
        fd = (fp - fm) / (2 * eps)
        np.testing.assert_allclose(K @ dirn, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())


def test_jacobian_is_symmetric_negative_semidefinite_and_translation_free():
    c, x, v = _cloth(rows=4, cols=4, scale=0.97)             # compressed: the clamp is active
    K = oracle.stiffness(c, x).toarray()
    assert np.abs(K - K.T).max() <= 1e-12 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).max() <= 1e-9 * np.abs(K).max()
    t = np.tile([0.3, -0.2, 0.7], x.size // 3)
    assert np.abs(K @ t).max() <= 1e-12 * np.abs(K).max()


def test_free_cloth_keeps_its_momentum():
    c, x, v = _cloth(rows=6, cols=7)
    x1, v1 = oracle.implicit_step(dict(c, dt=wl.f32(1e-3)), x, v, steps=3)
    np.testing.assert_allclose(v1.reshape(-1, 3).sum(0), v.reshape(-1, 3).sum(0), rtol=0,
                               atol=1e-12 * np.abs(v).sum())


def test_agrees_with_the_explicit_step_to_third_order():
    c, x, v = _cloth(p=0.4, drag=0.01, g=(0.0, 0.0, -9.81))
    errs = []
    for h in (4e-4, 2e-4, 1e-4):
        ch = dict(c, dt=h)
        xi, _ = oracle.implicit_step(ch, x, v, pins=[0, 5])
        xe, _ = oracle.step(ch, x, v, pins=[0, 5], steps=1)
        errs.append(np.abs(xi - xe).max())
    assert errs[0] / errs[1] > 6.0 and errs[1] / errs[2] > 6.0, errs
