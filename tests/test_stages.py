"""Host logic of the training stages (Sec. 3.2.1, Table 1, Sec. 5) against
the oracle: the group tables, the blob scaling, the schedules, the freeze
masks, and the differential-evolution engine step for step (same draws, same
FP64 objective: bit-identical populations)."""
import numpy as np
import pytest

import oracle
from paper_2403_12820_gb300 import stages
from paper_2403_12820_gb300 import workloads as wl


@pytest.mark.parametrize("cell", ["cnn", "pcell"])
def test_groups_match_the_oracle_tables(cell):
    ref = oracle.CNN_GROUPS if cell == "cnn" else oracle.PCELL_GROUPS
    assert [tuple(g) for g in stages.scale_groups(cell)] == [tuple(g) for g in ref]


@pytest.mark.parametrize("cell,n", [("cnn", 13036), ("pcell", 40)])
def test_scaled_blob_matches_the_oracle(cell, n):
    rng = np.random.default_rng(1)
    w0 = rng.normal(size=n).astype(np.float32)
    x = rng.uniform(-4, 4, size=6)
    got = stages.scaled(w0, cell, x)
    ref = oracle.scaled_blob(w0.astype(np.float64), cell, x)
    assert got.dtype == np.float32
    assert np.array_equal(got, ref.astype(np.float32))


def test_freeze_masks():
    m = stages.freeze_mask("cnn", ["WL", "bL"], 13027)
    assert m.dtype == np.uint8 and m.sum() == 864 + 3 and m[10944:11811].all()
    ref = oracle.group_mask(13027, "cnn", ["WD", "P"])
    assert np.array_equal(stages.freeze_mask("cnn", ["WD", "P"], 13027).astype(bool), ref)
    p = stages.freeze_mask("pcell", ["N_near", "b_L"], 39)
    assert p.sum() == 8 + 3 and p[12:20].all() and p[36:39].all()
    with pytest.raises(ValueError):
        stages.freeze_mask("pcell", ["bL"], 39)


def test_schedules_match_the_oracle():
    s = stages.StepLR(1e-2, 25, 0.5)
    c = stages.CosineLR(1e-3, 1e-6, 200)
    for t in range(0, 260):
        assert s(t) == pytest.approx(oracle.lr_step(1e-2, 25, 0.5, t), rel=1e-15)
        assert c(t) == pytest.approx(oracle.lr_cosine(1e-3, 1e-6, 200, min(t, 200)), rel=1e-15)
    with pytest.raises(ValueError):
        stages.StepLR(1e-3, 0, 0.5)


@pytest.mark.parametrize("F,CR,first", [(0.5, 0.9, None), (0.8, 0.2, True), (0.0, 1.0, None), (1.2, 0.0, True)])
def test_de_engine_is_step_for_step_the_oracle(F, CR, first):
    rng = np.random.default_rng(7)
    A = rng.normal(size=(5, 5))
    f = lambda z: float(np.cos(3 * z).sum() + 0.2 * z @ A @ z)
    lo, hi = -np.ones(5) * 2, np.ones(5) * 3
    d = wl.de_draws(seed=21, pop=11, dim=5, generations=12)
    x0 = np.full(5, 0.25) if first else None
    got = stages.differential_evolution(f, lo, hi, d, F=F, CR=CR, first=x0)
    bx, bf, hist, pop, fit, evals = oracle.de_minimize(f, lo, hi, d, F=F, CR=CR, first=x0)
    assert np.array_equal(got["population"], pop) and np.array_equal(got["fitness"], fit)
    assert got["history"] == hist and got["f"] == bf and np.array_equal(got["x"], bx)
    assert got["evals"] == evals == 11 * 13


def test_de_engine_skips_non_finite_trials():
    calls = []

    def f(z):
        calls.append(1)
        return np.inf if z[0] > 0.5 else float((z * z).sum())

    d = wl.de_draws(seed=2, pop=6, dim=2, generations=4)
    res = stages.differential_evolution(f, [-1, -1], [1, 1], d, first=np.zeros(2))
    assert res["f"] == 0.0 and np.isfinite(res["fitness"]).sum() >= 1
    assert len(calls) == res["evals"]
