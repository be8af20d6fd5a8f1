"""Pins of the larger-step physics target (Sec. 5's larger-step
integration): the mean acceleration over one plain step is the plain step's
acceleration without pressure; over k steps it is the average of the k
per-step accelerations."""
import numpy as np

import oracle
from paper_2403_12820_gb300 import workloads as wl


def _cloth():
    rng = np.random.default_rng(21)
    c = wl.cloth_spec(6, 7, p=0.3)
    x, v = wl.sag_state(c, rng, amp=0.01, vamp=0.05)
    return c, x.astype(np.float64), v.astype(np.float64)


def test_one_step_mean_acceleration_is_the_force_over_mass():
    c, x, v = _cloth()
    pins = [0, 6]
    got = oracle.mean_accel(c, x, v, pins, k=1)
    ref = (oracle.total_force(c, x, v) - oracle.pressure_force(c, x)) / c["m"]
    free = (1 - oracle.pin_mask(c, pins)).reshape(6, 7).astype(bool)
    np.testing.assert_allclose(got[free], ref[free], rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_k_step_mean_is_the_average_of_the_step_accelerations():
    c, x, v = _cloth()
    k = 5
    accs, xt, vt = [], x, v
    for _ in range(k):
        accs.append(oracle.total_force(c, xt, vt) / c["m"])
        xt, vt = oracle.step(c, xt, vt, steps=1)
    ref = np.mean(accs, axis=0) - oracle.pressure_force(c, x) / c["m"]
    got = oracle.mean_accel(c, x, v, (), k=k)
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
