"""Pins of the oracle's training stages (Sec. 3.2.1, Table 1, Sec. 5):
differential evolution against textbook optima and its special cases, the
learning-rate schedules against torch's schedulers, the masked Adam update
against the unmasked one and torch.optim.Adam, and the group tables against
the cells' own blob layouts (through the oracle's forward passes)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2403_12820_gb300 import workloads as wl

pytestmark = pytest.mark.filterwarnings("ignore::UserWarning")


# ------------------------------------------------------------ draws (inputs)
def test_de_draws_are_valid():
    d = wl.de_draws(seed=3, pop=9, dim=4, generations=7)
    assert d["init"].shape == (9, 4) and (d["init"] >= 0).all() and (d["init"] < 1).all()
    for g in range(7):
        for i in range(9):
            r = [int(k) for k in d["idx"][g, i]]
            assert len(set(r + [i])) == 4 and all(0 <= k < 9 for k in r)
    assert d["jrand"].min() >= 0 and d["jrand"].max() < 4
    assert d["cross"].shape == (7, 9, 4)
    with pytest.raises(ValueError):
        wl.de_draws(pop=3)


# ------------------------------------------------------------ DE/rand/1/bin
def test_de_sphere_converges_to_the_origin():
    d = wl.de_draws(seed=11, pop=20, dim=3, generations=150)
    x, f, hist, pop, fit, evals = oracle.de_minimize(lambda z: float((z * z).sum()), [-5] * 3, [5] * 3, d,
                                                     F=0.5, CR=0.9)
    assert f < 1e-10 and np.abs(x).max() < 1e-5
    assert evals == 20 * 151


def test_de_rosenbrock_finds_its_minimum():
    rosen = lambda z: float(100.0 * (z[1] - z[0] ** 2) ** 2 + (1.0 - z[0]) ** 2)
    d = wl.de_draws(seed=5, pop=24, dim=2, generations=300)
    x, f, *_ = oracle.de_minimize(rosen, [-2, -2], [2, 2], d, F=0.6, CR=0.9)
    assert f < 1e-6 and np.abs(x - 1.0).max() < 2e-3


def test_de_best_is_monotone_and_the_population_stays_in_the_box():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(4, 4))
    f = lambda z: float(np.sin(z).sum() + z @ A @ z * 0.1)
    d = wl.de_draws(seed=8, pop=10, dim=4, generations=30)
    lo, hi = np.array([-1.0, -2, -3, 0]), np.array([1.0, 0, 3, 0.5])
    x, fb, hist, pop, fit, _ = oracle.de_minimize(f, lo, hi, d, F=0.9, CR=0.5)
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    assert (pop >= lo).all() and (pop <= hi).all()
    assert fb == min(fit) == hist[-1]
    for i in range(10):
        assert fit[i] == f(pop[i])


def test_de_with_F0_CR1_selects_between_member_and_r1():
    """F = 0 and CR = 1 make every trial the member r1: one generation keeps,
    for each i, the better of x_i and x_r1 (old population, ties to r1)."""
    rng = np.random.default_rng(4)
    c = rng.normal(size=3)
    f = lambda z: float(((z - c) ** 2).sum())
    d = wl.de_draws(seed=9, pop=8, dim=3, generations=1)
    lo, hi = -np.ones(3) * 3, np.ones(3) * 3
    start = lo + d["init"] * (hi - lo)
    _, _, _, pop, fit, _ = oracle.de_minimize(f, lo, hi, d, F=0.0, CR=1.0)
    for i in range(8):
        r1 = int(d["idx"][0, i, 0])
        want = start[r1] if f(start[r1]) <= f(start[i]) else start[i]
        assert np.array_equal(pop[i], want)


def test_de_with_CR0_changes_only_the_forced_component():
    d = wl.de_draws(seed=12, pop=6, dim=5, generations=1)
    lo, hi = -np.ones(5) * 10, np.ones(5) * 10
    start = lo + d["init"] * (hi - lo)
    seen = []
    f = lambda z: (seen.append(np.array(z)), -1.0)[1] if len(seen) >= 6 else (seen.append(np.array(z)), 0.0)[1]
    oracle.de_minimize(f, lo, hi, d, F=0.5, CR=0.0)
    trials = seen[6:]
    for i in range(6):
        diff = np.nonzero(trials[i] != start[i])[0]
        assert set(diff.tolist()) <= {int(d["jrand"][0, i])}


def test_de_first_member_is_kept_when_it_is_the_optimum():
    c = np.array([0.3, -0.7])
    f = lambda z: float(((z - c) ** 2).sum())
    d = wl.de_draws(seed=1, pop=6, dim=2, generations=5)
    x, fb, *_ = oracle.de_minimize(f, [-1, -1], [1, 1], d, F=0.5, CR=0.9, first=c)
    assert fb == 0.0 and np.array_equal(x, c)


# ------------------------------------------------------------ schedules
def _torch_lrs(sched_ctor, lr0, n):
    p = torch.nn.Parameter(torch.zeros(1, dtype=torch.float64))
    opt = torch.optim.SGD([p], lr=lr0)
    sch = sched_ctor(opt)
    out = []
    for _ in range(n):
        out.append(opt.param_groups[0]["lr"])
        opt.step()
        sch.step()
    return out


def test_step_schedule_matches_torch():
    ref = _torch_lrs(lambda o: torch.optim.lr_scheduler.StepLR(o, step_size=7, gamma=0.3), 1e-2, 40)
    got = [oracle.lr_step(1e-2, 7, 0.3, t) for t in range(40)]
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=0)


def test_cosine_schedule_matches_torch_and_its_end_points():
    ref = _torch_lrs(lambda o: torch.optim.lr_scheduler.CosineAnnealingLR(o, T_max=50, eta_min=1e-5), 1e-3, 51)
    got = [oracle.lr_cosine(1e-3, 1e-5, 50, t) for t in range(51)]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    assert got[0] == 1e-3 and abs(got[50] - 1e-5) < 1e-20
    for t in range(51):   # symmetric about the midpoint of the two ends
        assert abs(got[t] + got[50 - t] - (1e-3 + 1e-5)) < 1e-18
    assert all(b < a for a, b in zip(got, got[1:]))


# ------------------------------------------------------------ masked Adam
def test_masked_adam_matches_unmasked_on_trainable_entries_and_freezes_the_rest():
    rng = np.random.default_rng(6)
    n = 40
    th, g, m, v = rng.normal(size=n), rng.normal(size=n), rng.normal(size=n) * 0.1, rng.random(n) * 0.1
    mask = rng.random(n) < 0.5
    t1, m1, v1 = oracle.adam_step_masked(th, g, m, v, t=5, lr=1e-3, mask=mask)
    t2, m2, v2 = oracle.adam_step(th, g, m, v, t=5, lr=1e-3)
    assert np.array_equal(t1[mask], t2[mask]) and np.array_equal(m1[mask], m2[mask])
    assert np.array_equal(v1[mask], v2[mask])
    assert np.array_equal(t1[~mask], th[~mask]) and np.array_equal(m1[~mask], m[~mask])
    assert np.array_equal(v1[~mask], v[~mask])


def test_masked_adam_against_torch_adam():
    rng = np.random.default_rng(10)
    n = 30
    th0 = rng.normal(size=n)
    mask = np.arange(n) % 3 != 0
    p = torch.nn.Parameter(torch.tensor(th0[mask]))
    opt = torch.optim.Adam([p], lr=2e-3, betas=(0.9, 0.999), eps=1e-8)
    th, m, v = th0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        g = rng.normal(size=n)
        p.grad = torch.tensor(g[mask])
        opt.step()
        th, m, v = oracle.adam_step_masked(th, g, m, v, t=t, lr=2e-3, mask=mask)
    np.testing.assert_allclose(th[mask], p.detach().numpy(), rtol=1e-13, atol=1e-15)
    assert np.array_equal(th[~mask], th0[~mask])


# ------------------------------------------------------------ group tables
def test_group_tables_follow_the_blob_layouts():
    C = 32
    sizes = {"W1": C * 6 * 9, "W2": C * C * 9, "WL": 3 * C * 9, "P": C * C, "WN": 3 * C, "WD": 3 * C}
    prev = 0
    for name, a, b in oracle.CNN_GROUPS:
        assert b - a == sizes[name] and a >= prev
        prev = b
    covered = oracle.group_mask(oracle.N_PARAMS, "cnn", [g[0] for g in oracle.CNN_GROUPS])
    assert covered.sum() == oracle.N_PARAMS - 3          # all trainable weights but bL
    pm = oracle.group_mask(oracle.PCELL_BLOB, "pcell", [g[0] for g in oracle.PCELL_GROUPS])
    assert pm[:36].all() and not pm[36:].any()
    with pytest.raises(AssertionError):
        oracle.group_mask(10, "pcell", ["nope"])


def _cloth(n=6):
    rng = np.random.default_rng(3)
    c = wl.cloth_spec(n, n + 1, p=0.3)
    x, v = wl.sag_state(c, rng, amp=0.02, vamp=0.1)
    return c, x.astype(np.float64), v.astype(np.float64)


def test_scaling_every_pcell_group_scales_the_bias_free_cell():
    """With b_L = 0 the literal cell's output is linear in (w_L, w_N, w_D)
    jointly: the same factor on all six groups scales it."""
    c, x, v = _cloth()
    w = wl.pcell_blob(2005, h=c["h"]).astype(np.float64)
    w[36:39] = 0.0
    rng = np.random.default_rng(1)
    w[12:36] = rng.normal(size=24)
    a = oracle.pcell_accel(w, c, x, v)
    a3 = oracle.pcell_accel(oracle.scaled_blob(w, "pcell", [-2.5] * 6), c, x, v)
    np.testing.assert_allclose(a3, -2.5 * a, rtol=1e-12, atol=1e-12 * np.abs(a).max())
    # one group at a time: far-tap weights of the linear branch enter linearly
    wl_only = w.copy(); wl_only[12:36] = 0.0
    base = oracle.pcell_accel(wl_only, c, x, v)
    far = wl_only.copy(); far[0:8] = 0.0
    a_far = oracle.pcell_accel(far, c, x, v)
    got = oracle.pcell_accel(oracle.scaled_blob(wl_only, "pcell", [1, 3, 1, 1, 1, 1]), c, x, v)
    np.testing.assert_allclose(got, base + 2.0 * a_far, rtol=1e-12, atol=1e-12 * np.abs(base).max())


def test_scaling_the_cnn_output_layers_scales_the_cell():
    """With bL = 0 the C-cell output is linear in (WL, WN, WD) jointly, and
    scaling W1 by s and W2 by 1/s leaves it unchanged (the trunk is linear)."""
    c, x, v = _cloth()
    w = wl.kaiming_blob(2003, in_scale=(1.0 / c["h"],) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3).astype(np.float64)
    w[11808:11811] = 0.0
    a = oracle.net_accel(w, c, x, v)
    got = oracle.net_accel(oracle.scaled_blob(w, "cnn", [1, 1, 0.5, 1, 0.5, 0.5]), c, x, v)
    np.testing.assert_allclose(got, 0.5 * a, rtol=1e-10, atol=1e-12 * np.abs(a).max())
    got = oracle.net_accel(oracle.scaled_blob(w, "cnn", [4.0, 0.25, 1, 1, 1, 1]), c, x, v)
    np.testing.assert_allclose(got, a, rtol=1e-10, atol=1e-12 * np.abs(a).max())
