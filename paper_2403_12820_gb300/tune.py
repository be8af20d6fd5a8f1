"""Launch-shape autotuner of the plain step, with a JSON cache.

The plain step runs a batch of cloths of uneven sizes in one persistent
launch; how the (cloth, 120-column strip, row segment) work list is cut and
how many warps share it decides how well the launch fills the GPU.  The
timing itself runs in libcloth (`cloth_tune_launch`: CUDA events around plain
steps that write only the spare state buffer, so the state does not move).
This module chooses the candidates, keys each result by kernel, GPU and
batch shape, and keeps it in a JSON file, so that a batch of the same shape
on the same kind of GPU is set up again without timing.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

# Candidates (seg_rows, warps_per_sm), in cloth_set_launch's terms: seg_rows
# >= 4 cuts the strips into segments of that many rows (one warp per segment
# by default), -1 gives balanced row shares; warps_per_sm -1 is the default.
DEFAULT_CANDIDATES: tuple[tuple[int, int], ...] = (
    (8, -1), (12, -1), (16, -1), (20, -1), (24, -1), (28, -1), (30, -1), (32, -1), (34, -1), (36, -1), (40, -1),
    (48, -1), (64, -1),
    (-1, -1), (-1, 8), (-1, 16),
)
MIN_SEG_ROWS = 4


def validate(candidates) -> list[tuple[int, int]]:
    """The candidates as (int, int) pairs; ValueError for an empty list or one
    outside cloth_set_launch's ranges."""
    out = []
    for c in candidates:
        R, w = int(c[0]), int(c[1])
        if not (R == -1 or R >= MIN_SEG_ROWS):
            raise ValueError(f"seg_rows {R}: must be -1 or >= {MIN_SEG_ROWS}")
        if not (w == -1 or 1 <= w <= 64):
            raise ValueError(f"warps_per_sm {w}: must be -1 or 1..64")
        out.append((R, w))
    if not out:
        raise ValueError("no candidates")
    return out


def kernel_name(specs) -> str:
    """The plain-step kernel a batch runs: spring-axis damping (mu != 0) in any
    cloth selects the damped variant."""
    return "plain_step_damp" if any(float(s.get("mu", 0.0)) != 0.0 for s in specs) else "plain_step"


def batch_key(kernel: str, device: str, sm_count: int, grids) -> str:
    """Cache key: the kernel, the GPU model and SM count, and the ordered list
    of grid sizes (the work list depends only on these)."""
    shape = [[int(r), int(c)] for r, c in grids]
    digest = hashlib.sha256(json.dumps([kernel, device, int(sm_count), shape]).encode()).hexdigest()[:20]
    return f"{kernel}/{int(sm_count)}sm/{len(shape)}x/{digest}"


def pick(candidates, us) -> int:
    """Index of the fastest candidate (the first of equal times)."""
    if len(candidates) != len(us) or not us:
        raise ValueError("one time per candidate")
    best = 0
    for i, t in enumerate(us):
        if t < us[best]:
            best = i
    return best


class LaunchCache:
    """A JSON file mapping batch keys to tuned launch shapes."""

    def __init__(self, path: str):
        self.path = path
        self.data: dict = {}
        if os.path.exists(path):
            with open(path) as fh:
                data = json.load(fh)
            if not isinstance(data, dict):
                raise ValueError(f"{path}: not a launch cache")
            self.data = data

    def get(self, key: str) -> dict | None:
        rec = self.data.get(key)
        if rec is None:
            return None
        validate([(rec["seg_rows"], rec["warps_per_sm"])])
        return rec

    def put(self, key: str, record: dict) -> None:
        self.data[key] = record
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, suffix=".tmp")
        with os.fdopen(fd, "w") as fh:
            json.dump(self.data, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def autotune(cb, cache_path: str | None = None, candidates=DEFAULT_CANDIDATES, warmup: int = 3, steps: int = 20,
             retune: bool = False) -> dict:
    """Pick the plain step's launch shape for the ClothBatch `cb` and apply it.

    With a cache file holding this batch's key (and retune False) the stored
    shape is applied without timing.  Otherwise every candidate is timed by
    libcloth and the fastest is applied (and stored when a cache path is
    given).  Returns the record: seg_rows, warps_per_sm, us_per_step, the
    timed candidates, and whether it came from the cache."""
    import torch

    cands = validate(candidates)
    props = torch.cuda.get_device_properties(cb.device)
    key = batch_key(kernel_name(cb.specs), props.name, props.multi_processor_count,
                    [(s["rows"], s["cols"]) for s in cb.specs])
    cache = LaunchCache(cache_path) if cache_path else None
    if cache is not None and not retune:
        rec = cache.get(key)
        if rec is not None:
            cb.set_launch(int(rec["seg_rows"]), int(rec["warps_per_sm"]))
            return dict(rec, key=key, cached=True)
    best, us = cb.tune_launch(cands, warmup=warmup, steps=steps)
    if best != pick(cands, us):
        raise RuntimeError("libcloth applied a different candidate than the fastest timed")
    rec = {"seg_rows": cands[best][0], "warps_per_sm": cands[best][1], "us_per_step": us[best],
           "candidates": [[R, w, t] for (R, w), t in zip(cands, us)], "warmup": int(warmup), "steps": int(steps)}
    if cache is not None:
        cache.put(key, rec)
    return dict(rec, key=key, cached=False)


def net_tile_choices(precision: int) -> list[dict]:
    """Tile shapes of the network step for networks of `precision`
    (cloth_net_tile_choices): per choice its output rows, columns and kind
    ("cuda" cores or "tensor" cores); the first is the default."""
    import ctypes

    from . import _lib
    rows, cols, kinds = (ctypes.c_int32 * 16)(), (ctypes.c_int32 * 16)(), (ctypes.c_int32 * 16)()
    n = ctypes.c_int32()
    _lib.call("cloth_net_tile_choices", int(precision), rows, cols, kinds, 16, ctypes.byref(n))
    return [{"rows": int(rows[i]), "cols": int(cols[i]), "kind": "tensor" if kinds[i] else "cuda"}
            for i in range(min(16, n.value))]


def autotune_net(cb, net, cache_path: str | None = None, warmup: int = 3, steps: int = 10,
                 retune: bool = False) -> dict:
    """Pick the network step's tile shape for the ClothBatch `cb` and the Net
    `net` (in its precision) and apply it, as autotune does for the plain
    step: from the cache when it holds this batch's key, else timed by
    libcloth (cloth_tune_net).  Returns the record: the choice index, its
    shape, us_per_step, the timed choices, and whether it came from the
    cache."""
    import torch

    props = torch.cuda.get_device_properties(cb.device)
    key = batch_key(f"net_step_p{int(net.precision)}", props.name, props.multi_processor_count,
                    [(s["rows"], s["cols"]) for s in cb.specs])
    cache = LaunchCache(cache_path) if cache_path else None
    choices = net_tile_choices(net.precision)
    if cache is not None and not retune:
        rec = cache.data.get(key)
        if rec is not None:
            if not 0 <= int(rec["choice"]) < len(choices) or choices[int(rec["choice"])] != rec["shape"]:
                raise ValueError(f"cached tile shape {rec['shape']} is not a choice")
            cb.set_net_tile(net.precision, int(rec["choice"]))
            return dict(rec, key=key, cached=True)
    best, us = cb.tune_net(net, warmup=warmup, steps=steps)
    if best != pick(list(range(len(choices))), us):
        raise RuntimeError("libcloth applied a different tile shape than the fastest timed")
    rec = {"choice": best, "shape": choices[best], "us_per_step": us[best],
           "candidates": [[ch, t] for ch, t in zip(choices, us)], "warmup": int(warmup), "steps": int(steps)}
    if cache is not None:
        cache.put(key, rec)
    return dict(rec, key=key, cached=False)
