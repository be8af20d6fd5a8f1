#!/usr/bin/env python
"""Throughput benchmark: cloth node-steps/s on one GB300.

Default workload (`plain_batch`): 64 square cloths with sides U{64..512}
(5.97M nodes, seed 1002), k x U(0.8, 1.2), 1-4 pinned boundary nodes,
pressure ~ N(0, 0.5) N/m^2 per cloth, FP32, every step one batched launch,
replayed from captured CUDA graphs.  One bench step = one plain step of the
whole batch.  The 306 MB double-buffered state is larger than the 129 MB L2,
so no flush is needed between steps.

`--impl reference` times the FP64 CPU oracle on the same workload instead
(bounded sample, host cores); under torchrun only rank 0 runs it.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

BYTES_PER_NODE_STEP = 48       # read u, v (24 B) + write u, v (24 B), FP32
PLAIN_SOURCES = ["paper_2403_12820_gb300/csrc/plain_step.cu", "paper_2403_12820_gb300/csrc/cloth_internal.cuh"]
CLOCK_FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


# ------------------------------------------------------------------ helpers
def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40000)
    p.add_argument("--warmup", type=int, default=400)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--graph-chunk", type=int, default=100)
    p.add_argument("--no-tune", action="store_true", help="keep the default launch shape (no autotuning)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cnn", action="store_true")
    p.add_argument("--cnn-steps", type=int, default=1000)
    p.add_argument("--no-mixed", action="store_true")
    p.add_argument("--mixed-steps", type=int, default=5000)
    p.add_argument("--no-train", action="store_true")
    p.add_argument("--no-pcell", action="store_true")
    p.add_argument("--no-larger-step", action="store_true")
    p.add_argument("--train-iters", type=int, default=20)
    p.add_argument("--de-generations", type=int, default=6)
    p.add_argument("--bf16-tile", type=int, default=0,
                   help="cnn_step section: tile choice of the BF16 network step (tune.net_tile_choices)")
    p.add_argument("--fp32-tile", type=int, default=0,
                   help="cnn_step section: tile choice of the FP32 network step (tune.net_tile_choices)")
    p.add_argument("--only", choices=["cnn", "cnn_step", "mixed", "pcell", "larger_step", "train", "single_cloth"],
                   default=None,
                   help="run one section alone and print its JSON (for profiling; not a bench line)")
    return p.parse_args(argv)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


FP32_LANES_PER_SM = 128   # FP32 FMA lanes of one SM (4 schedulers x 32)


def fp32_alu_peak(dev):
    """CUDA-core FP32 peak in TFLOP/s from the unit counts and the maximum SM
    clock: SMs x 128 FMA lanes x 2 flop x clock."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        idx = torch.cuda.current_device() if dev is None else torch.device(dev).index or 0
        r = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits", "-i", str(idx)],
                           capture_output=True, text=True, timeout=20)
        mhz = float(r.stdout.strip().splitlines()[0])
    except Exception:
        pass
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, sms, mhz


def kernel_hash(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(name: str, src_files, units: float):
    """DRAM bytes per launch from the committed ncu summary, scaled to `units`
    nodes; None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", f"{name}.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        if d.get("source_hash") != kernel_hash(src_files):
            return None
        return float(d["dram_bytes_per_node"]) * units
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms for one GPU."""

    def __init__(self, device_index: int):
        import torch
        self.samples = []
        self.proc = None
        try:
            pr = torch.cuda.get_device_properties(device_index)
            bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
        except Exception:
            bus = str(device_index)
        self.bus = bus

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", self.bus], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def mark(self):
        return time.time()

    def stop(self, t0: float, t1: float) -> dict:
        time.sleep(0.25)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()
        sel = [p for (t, p) in self.samples if t0 - 0.25 <= t <= t1 + 0.25] or [p for (_, p) in self.samples]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for p in sel if num(p[1]) is not None]
        smax = [num(p[2]) for p in sel if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in sel for i in range(4) if p[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(sel)}


def dist_setup(gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Largest value over all ranks (the slowest rank sets the job time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle
def _oracle_cloth_steps(args):
    spec, pins, x, v, steps = args
    import oracle
    t = time.perf_counter()
    oracle.step(spec, x, v, pins=pins, steps=steps)
    return time.perf_counter() - t


def oracle_plain_rate(cfg, steps: int, cores: int):
    """Node-steps/s of the FP64 oracle over all cloths of `cfg` for `steps`
    steps, cloths spread over a spawn pool of `cores` processes."""
    import oracle
    oracle.build()
    jobs = [(s, p, x, v, steps) for s, p, x, v in zip(cfg["specs"], cfg["pins"], cfg["x"], cfg["v"])]
    jobs.sort(key=lambda j: -j[0]["rows"] * j[0]["cols"])
    nodes = sum(s["rows"] * s["cols"] for s in cfg["specs"])
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_cloth_steps, jobs[:cores], chunksize=1)     # warm the workers
        t = time.perf_counter()
        pool.map(_oracle_cloth_steps, jobs, chunksize=1)
        wall = time.perf_counter() - t
    return nodes * steps / wall, wall


def oracle_single_rates():
    """Single-thread FP64 oracle rates: the plain step on the batch's largest
    cloth (4 steps) and the C-cell network step on one 128 x 128 cloth."""
    import numpy as np

    import oracle
    from paper_2403_12820_gb300 import workloads as wl
    cfg = wl.plain_batch()
    b = max(range(len(cfg["specs"])), key=lambda i: cfg["specs"][i]["rows"] * cfg["specs"][i]["cols"])
    s = cfg["specs"][b]
    t = time.perf_counter()
    oracle.step(s, cfg["x"][b], cfg["v"][b], pins=cfg["pins"][b], steps=4)
    plain = s["rows"] * s["cols"] * 4 / (time.perf_counter() - t)
    cc = wl.cnn_batch(count=1)
    w = cnn_blob(cc["specs"][0]["h"]).astype(np.float64)
    t = time.perf_counter()
    oracle.net_step(w, cc["specs"][0], cc["x"][0], cc["v"][0], pins=cc["pins"][0], steps=1)
    cnn = cc["specs"][0]["rows"] * cc["specs"][0]["cols"] / (time.perf_counter() - t)
    sc = wl.single_cloth(n=32)
    t = time.perf_counter()
    oracle.step(sc["specs"][0], sc["x"][0], sc["v"][0], pins=sc["pins"][0], steps=2000)
    single_us = (time.perf_counter() - t) / 2000 * 1e6
    return {"single_thread_plain_node_steps_per_s": plain,
            "single_cloth_32x32_us_per_step": single_us,
            "single_thread_cnn_node_steps_per_s": cnn,
            "single_thread_sample": f"plain: one {s['rows']} x {s['cols']} cloth x 4 steps; "
                                    "C-cell network step: one 128 x 128 cloth x 1 step; "
                                    "single cloth: 32 x 32 x 2000 steps"}


# ------------------------------------------------------------------ runs
def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2403_12820_gb300 import workloads as wl
    cfg = wl.plain_batch()
    cores = os.cpu_count() or 1
    nodes = sum(s["rows"] * s["cols"] for s in cfg["specs"])
    sample_steps = 1
    # warm-up, then each timed bench step is one plain step of the whole batch
    steps = max(1, min(args.steps, 10))
    warm = max(0, min(args.warmup, 3))
    if warm:
        oracle_plain_rate(cfg, 1, cores)
    rate, wall = oracle_plain_rate(cfg, steps * sample_steps, cores)
    ms = wall / steps * 1e3
    return {
        "impl": "reference", "metric": "cloth node-steps/s (plain mass-spring step, batched cloths)",
        "value": rate, "unit": "node-steps/s", "n_gpus": args.gpus, "steps": steps, "warmup": warm,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "plain_batch: 64 cloths, sides U{64..512} (5.97M nodes), FP64 oracle on host cores",
                   "global_batch": 64, "nodes": nodes},
        "cpu_baseline": {"value": rate, "unit": "node-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"all 64 cloths x {steps} steps (bench steps capped at 10)"},
        "e2e": {"value": rate, "unit": "node-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_plain(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2403_12820_gb300 import shard
    from paper_2403_12820_gb300 import workloads as wl
    from paper_2403_12820_gb300.cloth import ClothBatch, pack

    # one batch of 64 cloths per rank (weak scaling), split over the ranks by
    # whole cloths, largest first (no data-path communication)
    cfg = wl.plain_batch(count=64 * world)
    job_nodes = sum(s["rows"] * s["cols"] for s in cfg["specs"])
    if world > 1:
        cfg = shard.take(cfg, shard.partition([s["rows"] * s["cols"] for s in cfg["specs"]], world)[rank])
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cb = ClothBatch(cfg["specs"], cfg["pins"], device=dev)
    x0 = pack(cfg["x"]).to(dev)
    v0 = pack(cfg["v"]).to(dev)
    cb.set_state(x0, v0)
    nodes = cb.total_nodes
    chunk = args.graph_chunk
    stream = torch.cuda.current_stream()

    # launch shape picked by the autotuner (untimed; the state does not move)
    if args.no_tune:
        seg, wps, _ = cb.get_launch()
        launch = {"seg_rows": seg, "warps_per_sm": wps, "tuned": False}
    else:
        from paper_2403_12820_gb300 import tune
        rec = tune.autotune(cb, candidates=tune.DEFAULT_CANDIDATES, warmup=3, steps=20)
        launch = {"seg_rows": rec["seg_rows"], "warps_per_sm": rec["warps_per_sm"], "tuned": True,
                  "candidates_us": {f"{R},{w}": round(t, 2) for R, w, t in rec["candidates"]}}

    cb.rollout(args.warmup, graph_chunk=chunk)
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(world)
    w0 = time.time()
    e0.record(stream)
    cb.rollout(args.steps, graph_chunk=chunk)
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    barrier(world)
    clocks = sampler.stop(w0, w1)
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world)
    status = cb.status()
    value = job_nodes * args.steps / (ms_max / 1e3)

    hbm, _, peak_kind = peaks()
    launch_s = ms / 1e3 / args.steps          # one plain-step kernel per step
    achieved = BYTES_PER_NODE_STEP * nodes / launch_s / 1e9
    traffic = ncu_traffic("plain_step_traffic", PLAIN_SOURCES, nodes)

    out = {
        "metric": "cloth node-steps/s (plain mass-spring step, batched cloths)",
        "value": value, "unit": "node-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "plain_batch: 64 cloths, sides U{64..512} (seed 1002), 5.97M nodes, FP32, "
                               f"CUDA graphs of {chunk} steps"
                               + (f"; {64 * world} cloths split over {world} ranks largest first" if world > 1 else ""),
                   "global_batch": 64 * world, "nodes_per_gpu": nodes, "job_nodes": job_nodes, "launch": launch,
                   "l2": "inputs larger than L2 (306 MB double-buffered state vs 129 MB L2)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "peak_kind": f"{peak_kind} (copy bandwidth)", "traffic": traffic,
                     "algorithmic_bytes_per_launch": BYTES_PER_NODE_STEP * nodes},
        # the plain-step kernel, and the kernel that sets the pinned nodes
        "gpu_launches": args.steps * (2 if any(len(p) for p in cfg["pins"]) else 1),
        "clocks": clocks,
        "status_word": status,
    }

    if not args.no_e2e:
        # end to end through the public API: pinned host state -> device,
        # a 100-step rollout, positions back to pinned host memory
        per_call = 100
        hx = torch.empty_like(x0, device="cpu").pin_memory()
        hv = torch.empty_like(v0, device="cpu").pin_memory()
        hx.copy_(x0); hv.copy_(v0)
        hout = torch.empty_like(hx).pin_memory()
        dx = torch.empty_like(x0); dv = torch.empty_like(v0)
        calls = max(1, min(20, args.steps // per_call))
        for _ in range(2):
            dx.copy_(hx, non_blocking=True); dv.copy_(hv, non_blocking=True)
            cb.set_state(dx, dv); cb.rollout(per_call, graph_chunk=per_call)
            xo, _ = cb.get_state(); hout.copy_(xo, non_blocking=True)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(calls):
            dx.copy_(hx, non_blocking=True); dv.copy_(hv, non_blocking=True)
            cb.set_state(dx, dv)
            cb.rollout(per_call, graph_chunk=per_call)
            xo, _ = cb.get_state()
            hout.copy_(xo, non_blocking=True)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, world)
        out["e2e"] = {"value": job_nodes * per_call * calls / el, "unit": "node-steps/s",
                      "h2d_bytes_per_step": (hx.numel() + hv.numel()) * 4 / per_call,
                      "d2h_bytes_per_step": hout.numel() * 4 / per_call,
                      "steps_per_call": per_call, "calls": calls}

    out["single_cloth"] = run_single_cloth(dev)
    if not args.no_cnn:
        out["cnn"] = run_cnn(args, dev)
    if not args.no_mixed:
        out["mixed_fallback"] = run_mixed(args, dev)
    if not args.no_pcell:
        out["pcell"] = run_pcell(args, dev, value / world)
    if not args.no_larger_step:
        out["larger_step"] = run_larger_step(args, dev, value / world)
    if not args.no_train:
        out["train"] = run_train(args, dev)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        rate, wall = oracle_plain_rate(cfg, 24, cores)
        out["cpu_baseline"] = {"value": rate, "unit": "node-steps/s", "cores": cores, "kind": "oracle",
                               "sample": f"all 64 cloths x 24 steps (143M node-steps), FP64 oracle, "
                                         f"{cores} processes, {wall:.1f} s wall"}
        out["cpu_baseline"].update(oracle_single_rates())
    cb.close()
    return out


CNN_FLOP_PER_NODE = 44480     # 22,240 MAC of the cell per node


def cnn_blob(h: float):
    from paper_2403_12820_gb300 import workloads as wl
    return wl.kaiming_blob(2003, in_scale=(1.0 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3)


def network_blob(h: float):
    """The trained C-cell weights committed with the package (the training
    run on the plain-simulator trajectories), else Kaiming weights; and
    whether they are the trained ones."""
    from paper_2403_12820_gb300.train import load_trained
    w = load_trained()
    return (w, True) if w is not None else (cnn_blob(h), False)


def run_cnn(args, dev):
    """Network step (Fig. 2) on 32 cloths of 128 x 128 drawn like the plain
    batch, from their state after 100 plain steps: node-steps/s of the BF16
    tensor-core step and of the FP32 CUDA-core step (trained weights), the
    ratio to the plain step on the same cloths, and the accuracy after 100
    steps against the plain step (Table 2's error: mean node distance over
    cloth width, and over the plain rollout's mean displacement) beside the
    gravity-only network (a = g) and the untrained Kaiming network."""
    import torch

    from paper_2403_12820_gb300 import workloads as wl
    from paper_2403_12820_gb300.cloth import ClothBatch, pack
    from paper_2403_12820_gb300.net import BF16, FP32, Net
    from paper_2403_12820_gb300.train import evaluate, gravity_only_blob

    cfg = wl.cnn_batch()
    h = cfg["specs"][0]["h"]
    blob, trained = network_blob(h)
    cp = ClothBatch(cfg["specs"], cfg["pins"], device=dev)
    cp.set_state(pack(cfg["x"]).to(dev), pack(cfg["v"]).to(dev))
    cp.rollout(100, graph_chunk=100)
    x0, v0 = cp.get_state()
    nodes = cp.total_nodes
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    cp.set_state(x0, v0)
    cp.rollout(10, graph_chunk=10)
    t_plain = timed(lambda k: cp.rollout(k, graph_chunk=100), 10 * args.cnn_steps)
    plain_rate = nodes * 10 * args.cnn_steps / t_plain
    _, bf16_peak, peak_kind = peaks()
    acc = evaluate({"bf16": (blob, BF16), "f32": (blob, FP32), "gravity_only": (gravity_only_blob(), FP32),
                    "untrained_kaiming_bf16": (cnn_blob(h), BF16)}, cfg, warm=100, steps=100, device=dev,
                   horizons=(300, 1000))
    zero = acc["gravity_only"]["error_rel_width"]
    out = {"workload": "cnn_batch: 32 cloths of 128 x 128 (524,288 nodes) drawn like the plain batch (seed 1003), "
                       f"from their state after 100 plain steps; {'trained' if trained else 'Kaiming'} weights",
           "trained": trained, "plain_same_cloths": plain_rate,
           "accuracy_100_steps": {"displacement_rel_width": acc["displacement_rel_width"],
                                  "gravity_only_error_rel_width": zero,
                                  "gravity_only_error_rel_displacement": acc["gravity_only"]["error_rel_displacement"],
                                  "untrained_kaiming_bf16_error_rel_width":
                                      acc["untrained_kaiming_bf16"]["error_rel_width"]}}
    def timed_segments(cn, fn, steps):
        """`steps` network steps as segments of 100 from the start state (a
        network rollout leaves the physical states after some hundreds of
        steps); CUDA events around each segment only."""
        total, left = 0.0, steps
        while left > 0:
            k = min(100, left)
            cn.set_state(x0, v0)
            total += timed(fn, k)
            left -= k
        return total

    tuned = {}
    for name, prec in (("bf16", BF16), ("f32", FP32)):
        net = Net(blob, prec, device=dev)
        cn = ClothBatch(cfg["specs"], cfg["pins"], device=dev)
        cn.set_state(x0, v0)
        # the step's tile shape from the launch tuner (the state does not move)
        from paper_2403_12820_gb300 import tune
        rec = tune.autotune_net(cn, net, warmup=3, steps=20)
        tuned[name] = rec["choice"]
        shape = lambda ch: f"{ch['rows']}x{ch['cols']} {ch['kind']}"
        tile = {"shape": shape(rec["shape"]), "candidates_us": {shape(ch): round(t, 2) for ch, t in rec["candidates"]}}
        cn.step_net(net, 3)
        steps = args.cnn_steps
        t = timed_segments(cn, lambda k: cn.step_net(net, k), steps)
        rate = nodes * steps / t
        tflops = CNN_FLOP_PER_NODE * rate / 1e12
        e = acc[name]
        out[name] = {"value": rate, "unit": "node-steps/s", "steps": steps, "ms_per_step": t / steps * 1e3,
                     "ratio_to_plain": rate / plain_rate, "error_100_steps_rel_width": e["error_rel_width"],
                     "error_100_steps_rel_displacement": e["error_rel_displacement"],
                     "error_rel_width_at_steps": e.get("horizon_errors"),
                     "beats_gravity_only": e["error_rel_width"] < zero,
                     "within_1pct_of_width": e["error_rel_width"] <= 0.01,
                     "achieved_tflops": tflops, "gpu_launches_per_step": 1, "timed_as": "segments of 100 steps",
                     "status_word": cn.status()}
        out[name]["tile"] = tile
        if prec == BF16 or rec["shape"]["kind"] == "tensor":
            out[name]["roofline"] = {"bound": "tensor", "achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                                     "frac": tflops / bf16_peak, "peak_kind": f"{peak_kind} (cuBLAS bf16 burst)",
                                     "algorithmic_flop_per_node": CNN_FLOP_PER_NODE}
        else:   # the FP32 step runs on the CUDA cores
            alu, sms, mhz = fp32_alu_peak(dev)
            out[name]["roofline"] = {"bound": "alu", "achieved": tflops, "peak": alu, "unit": "TFLOP/s",
                                     "frac": tflops / alu,
                                     "peak_kind": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {mhz:.0f} MHz",
                                     "algorithmic_flop_per_node": CNN_FLOP_PER_NODE}
        cn.close()
        net.close()
    # larger-step network: stride 4 (dt_net = 4 dt), 25 network steps cover the
    # simulated time of the 100 plain steps the error is taken against
    cp.set_state(x0, v0)
    cp.rollout(100, graph_chunk=100)
    xp, _ = cp.get_state()
    w = (cfg["specs"][0]["cols"] - 1) * h
    net = Net(blob, BF16, device=dev)
    cn = ClothBatch(cfg["specs"], cfg["pins"], device=dev)
    cn.set_net_tile(BF16, tuned["bf16"])   # the shape the tuner picked for these cloths
    cn.set_net_stride(4)
    cn.set_state(x0, v0)
    cn.step_net(net, 3)
    t = timed_segments(cn, lambda k: cn.step_net(net, k), args.cnn_steps)
    rate = nodes * args.cnn_steps / t
    cn.set_state(x0, v0)
    cn.step_net(net, 25)
    xn, _ = cn.get_state()
    err = (xn - xp).norm(dim=1).mean().item()
    out["bf16_stride4"] = {"value": rate, "unit": "node-steps/s (network steps of 4 dt)",
                           "plain_equivalent_node_steps_per_s": 4 * rate, "ratio_to_plain_equivalent": 4 * rate / plain_rate,
                           "error_100_plain_steps_rel_width": err / w, "status_word": cn.status(),
                           "note": "weights trained for steps of dt, run at 4 dt"}
    cn.close()
    net.close()
    cp.close()
    return out


def run_cnn_step(args, dev):
    """The BF16 and FP32 network steps alone on the network workload (no
    accuracy runs): `--cnn-steps` steps of each from the state after 100
    plain steps, for profiling."""
    import torch

    from paper_2403_12820_gb300 import workloads as wl
    from paper_2403_12820_gb300.cloth import ClothBatch, pack
    from paper_2403_12820_gb300.net import BF16, FP32, Net

    cfg = wl.cnn_batch()
    blob, trained = network_blob(cfg["specs"][0]["h"])
    cb = ClothBatch(cfg["specs"], cfg["pins"], device=dev)
    cb.set_state(pack(cfg["x"]).to(dev), pack(cfg["v"]).to(dev))
    cb.rollout(100, graph_chunk=100)
    x0, v0 = cb.get_state()
    out = {"trained": trained}
    for name, prec, tile in (("bf16", BF16, args.bf16_tile), ("f32", FP32, args.fp32_tile)):
        net = Net(blob, prec, device=dev)
        cb.set_net_tile(prec, tile)
        cb.set_state(x0, v0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        cb.step_net(net, args.cnn_steps)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"ms_per_step": e0.elapsed_time(e1) / max(1, args.cnn_steps), "steps": args.cnn_steps,
                     "tile_choice": tile, "status_word": cb.status()}
        net.close()
    cb.close()
    return out


def run_mixed(args, dev):
    """Large mixed batch with the plain-step fallback: 16 cloths with sides
    U{256..1024} falling onto a sphere, the BF16 network rollout (trained
    weights) captured in CUDA graphs, every 10th step judged by one plain
    step from the same state; a cloth whose largest node difference exceeds
    1e-3 m switches to the plain step.  Reports node-steps/s of the checked
    rollout over the configured 5000 steps and how many cloths switched, and
    (over 1000 steps) the unchecked network rollout and the plain rollout on
    the same cloths."""
    import torch

    from paper_2403_12820_gb300 import workloads as wl
    from paper_2403_12820_gb300.cloth import ClothBatch, pack
    from paper_2403_12820_gb300.net import BF16, Net

    cfg = wl.mixed_batch()
    h = cfg["specs"][0]["h"]
    x0, v0 = pack(cfg["x"]).to(dev), pack(cfg["v"]).to(dev)
    cb = ClothBatch(cfg["specs"], cfg["pins"], device=dev)
    nodes = cb.total_nodes
    blob, trained = network_blob(h)
    net = Net(blob, BF16, device=dev)
    from paper_2403_12820_gb300 import tune
    cb.set_state(x0, v0)
    tile_rec = tune.autotune_net(cb, net, warmup=2, steps=10)   # the network step's tile shape
    stream = torch.cuda.current_stream()
    steps = max(100, args.mixed_steps // 100 * 100)
    side = min(steps, 1000)

    def timed(fn, n):
        cb.set_state(x0, v0)
        cb.reset_modes()
        fn(100)                       # warm-up, graph capture
        cb.set_state(x0, v0)
        cb.reset_modes()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn(n)
        e1.record(stream)
        torch.cuda.synchronize()
        return nodes * n / (e0.elapsed_time(e1) / 1e3)

    checked = timed(lambda k: cb.rollout_net(net, k, check_every=10, residual_bound=1e-3, graph_chunk=100), steps)
    mode, resid = cb.modes()
    status = cb.status()
    xc, _ = cb.get_state()
    finite = bool(torch.isfinite(xc).all())
    # the same checked rollout again, untimed, in pieces of 500 steps: how
    # many cloths had switched to the plain step by then
    cb.set_state(x0, v0)
    cb.reset_modes()
    switched_by = {}
    for k in range(500, steps + 1, 500):
        cb.rollout_net(net, 500, check_every=10, residual_bound=1e-3, graph_chunk=100)
        switched_by[str(k)] = int(cb.modes()[0].sum().item())
    unchecked = timed(lambda k: cb.rollout_net(net, k, graph_chunk=100), side)
    plain = timed(lambda k: cb.rollout(k, graph_chunk=100), side)
    # the same rollouts with Coulomb contact (mu 0.3) in place of the
    # stopping contact, selected at run time (same graphs; this batch has no pins)
    for b in range(cb.B):
        cb.set_boundary(b, (0.0, 0.0, 0.0), 0.3)
    friction_net = timed(lambda k: cb.rollout_net(net, k, graph_chunk=100), side)
    friction_plain = timed(lambda k: cb.rollout(k, graph_chunk=100), side)
    out = {"workload": f"mixed_batch: 16 cloths, sides U{{256..1024}} (seed 1005), {nodes / 1e6:.2f}M nodes, "
                       f"sphere R = 0.3 w, BF16 network ({'trained' if trained else 'Kaiming'} weights), FP32 state",
           "trained": trained,
           "value": checked, "unit": "node-steps/s", "steps": steps, "check_every": 10, "residual_bound_m": 1e-3,
           "graph_chunk": 100, "switched_to_plain": int(mode.sum().item()), "cloths": cb.B,
           "switched_by_step": switched_by,
           "largest_residual_m": float(resid.max().item()), "state_finite": finite,
           "network_unchecked": unchecked, "plain_same_cloths": plain, "ratio_to_plain": checked / plain,
           "side_rollout_steps": side, "status_word": status,
           "coulomb_contact": {"network_unchecked": friction_net, "plain": friction_plain, "friction": 0.3},
           "gpu_launches_per_10_steps": 10 + 1 + 3 + 1,   # 10 network + 1 plain + residual, merge, latch + memset
           "tile": {"rows": tile_rec["shape"]["rows"], "cols": tile_rec["shape"]["cols"],
                    "candidates_us": [round(t, 2) for _, t in tile_rec["candidates"]]}}
    net.close()
    cb.close()
    return out


def run_single_cloth(dev):
    """One 32 x 32 cloth (the single-cloth workload: two corners pinned,
    1e-4 m noise), 2000 plain steps: a latency-bound case (the 24 KB state
    fits one SM), reported as microseconds per step (the CPU baseline times
    the oracle on it), with the paper's own step rates (100 x 100 cloths,
    other hardware) as context."""
    import torch

    from paper_2403_12820_gb300 import workloads as wl
    from paper_2403_12820_gb300.cloth import ClothBatch, pack

    from paper_2403_12820_gb300 import tune

    cfg = wl.single_cloth(n=32)
    cb = ClothBatch(cfg["specs"], cfg["pins"], device=dev)
    cb.set_state(pack(cfg["x"]).to(dev), pack(cfg["v"]).to(dev))
    rec = tune.autotune(cb, candidates=((4, -1), (8, -1), (16, -1), (32, -1), (-1, -1)), warmup=3, steps=50)
    cb.rollout(200, graph_chunk=100)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    cb.rollout(2000, graph_chunk=100)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) / 2000 * 1e3
    out = {"workload": "single_cloth: 32 x 32 (seed 1001), 2000 plain steps in CUDA graphs of 100",
           "us_per_step": us, "node_steps_per_s": 1024 / us * 1e6, "status_word": cb.status(),
           "launch": {"seg_rows": rec["seg_rows"], "warps_per_sm": rec["warps_per_sm"],
                      "candidates_us": {f"{R},{w}": round(t, 2) for R, w, t in rec["candidates"]}},
           "paper_context": {"nn_framework_node_steps_per_s": 2.32e6, "pbs_cpu_node_steps_per_s": 2.01e6,
                             "note": "Table 2: 232 and 201 steps/s on 100 x 100 cloths (RTX 2080 Ti; "
                                     "a CPU of unstated model)"}}
    cb.close()
    return out


def _ratio(a, b):
    """a / b, or None when the plain rate it is taken against was not
    measured (a section run alone)."""
    return None if b is None else a / b


def run_larger_step(args, dev, plain_rate: float | None):
    """Larger time steps on the 64-cloth plain batch (Sec. 5: larger-step and
    implicit integration): the implicit plain step (linearised backward
    Euler, 20 CG iterations) and the BF16 network step, both at 10 dt, in
    node-steps/s of their own steps and of the plain steps they stand for,
    and the implicit step's mean node distance to the explicit rollout after
    the same simulated time (100 plain steps), relative to cloth width."""
    import torch

    from paper_2403_12820_gb300 import workloads as wl
    from paper_2403_12820_gb300.cloth import ClothBatch, pack
    from paper_2403_12820_gb300.net import BF16, Net

    k, iters = 10, 20
    cfg = wl.plain_batch()
    x0, v0 = pack(cfg["x"]).to(dev), pack(cfg["v"]).to(dev)
    cb = ClothBatch(cfg["specs"], cfg["pins"], device=dev)
    nodes = cb.total_nodes
    stream = torch.cuda.current_stream()

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn(n)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    cb.set_state(x0, v0)
    cb.rollout(10 * k, graph_chunk=10 * k)
    xe, _ = cb.get_state()
    cb.set_state(x0, v0)
    cb.step_implicit(10, stride=k, cg_iters=iters)
    xi, _ = cb.get_state()
    widths = torch.tensor([(s["cols"] - 1) * s["h"] for s in cfg["specs"]], device=dev)
    err = torch.stack([(a - b).norm(dim=1).mean() for a, b in zip(cb.split(xi), cb.split(xe))]) / widths
    t_impl = timed(lambda n: cb.step_implicit(n, stride=k, cg_iters=iters), 10)
    impl_rate = nodes * 10 / t_impl
    # the explicit plain rollout again with every cloth's pins moving (0.05 m/s
    # along x), selected at run time: the moving-boundary path's cost
    cb.set_state(x0, v0)
    for b in range(cb.B):
        cb.set_boundary(b, (0.05, 0.0, 0.0), -1.0)
    cb.rollout(100, graph_chunk=100)
    t_mv = timed(lambda n: cb.rollout(n, graph_chunk=100), 1000)
    moving_rate = nodes * 1000 / t_mv
    for b in range(cb.B):
        cb.set_boundary(b, (0.0, 0.0, 0.0), -1.0)
    net = Net(network_blob(cfg["specs"][0]["h"])[0], BF16, device=dev)
    cn = ClothBatch(cfg["specs"], cfg["pins"], device=dev)
    cn.set_net_stride(k)
    cn.set_state(x0, v0)
    from paper_2403_12820_gb300 import tune
    net_tile = tune.autotune_net(cn, net, warmup=2, steps=10)["shape"]   # the state does not move
    cn.step_net(net, 3)
    t_net = timed(lambda n: cn.step_net(net, n), 50)
    net_rate = nodes * 50 / t_net
    out = {"workload": f"plain_batch: 64 cloths, sides U{{64..512}} (seed 1002), {nodes / 1e6:.2f}M nodes; "
                       f"steps of {k} dt",
           "stride": k,
           "implicit": {"value": impl_rate, "unit": "node-steps/s (implicit steps of 10 dt)", "cg_iters": iters,
                        "ms_per_step": t_impl / 10 * 1e3, "plain_equivalent_node_steps_per_s": k * impl_rate,
                        "ratio_to_explicit": _ratio(k * impl_rate, plain_rate),
                        "mean_error_rel_width_after_100_dt": float(err.mean().item()),
                        "max_cloth_error_rel_width": float(err.max().item()), "status_word": cb.status()},
           "bf16_network": {"value": net_rate, "unit": "node-steps/s (network steps of 10 dt)",
                            "ms_per_step": t_net / 50 * 1e3, "plain_equivalent_node_steps_per_s": k * net_rate,
                            "ratio_to_explicit": _ratio(k * net_rate, plain_rate), "status_word": cn.status(),
                            "tile": net_tile},
           "explicit_plain": plain_rate,
           "explicit_plain_moving_pins": {"value": moving_rate, "unit": "node-steps/s",
                                          "pin_velocity_m_s": [0.05, 0.0, 0.0]}}
    cb.close()
    cn.close()
    net.close()
    return out


def run_pcell(args, dev, plain_rate: float | None):
    """Network step with the literal cell (Eq. 6-7, Fig. 1: frozen difference
    channels, ISRU, three branches) on the plain batch's 64 cloths,
    spring-like weights (seed 2005): node-steps/s against the HBM roofline
    (48 B per node-step, as the plain step) and the ratio to the plain step."""
    import torch

    from paper_2403_12820_gb300 import workloads as wl
    from paper_2403_12820_gb300.cloth import ClothBatch, pack

    cfg = wl.plain_batch()
    cb = ClothBatch(cfg["specs"], cfg["pins"], device=dev)
    cb.set_state(pack(cfg["x"]).to(dev), pack(cfg["v"]).to(dev))
    nodes = cb.total_nodes
    w = torch.from_numpy(wl.pcell_blob()).to(dev)
    stream = torch.cuda.current_stream()
    cb.step_pcell(w, 20)
    steps = 400
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    cb.step_pcell(w, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    rate = nodes * steps / t
    hbm, _, peak_kind = peaks()
    achieved = BYTES_PER_NODE_STEP * rate / 1e9
    out = {"workload": "plain_batch cloths (5.97M nodes), literal cell with spring-like weights (seed 2005)",
           "value": rate, "unit": "node-steps/s", "steps": steps, "ms_per_step": t / steps * 1e3,
           "ratio_to_plain": _ratio(rate, plain_rate), "gpu_launches_per_step": 1, "status_word": cb.status(),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "peak_kind": f"{peak_kind} (copy bandwidth)",
                        "algorithmic_bytes_per_launch": BYTES_PER_NODE_STEP * nodes}}
    cb.close()
    return out


def run_train(args, dev):
    """Training iterations (Eq. 8, Table 1): 512 plain trajectories of 64 x 64
    x 200 steps kept on the device; each iteration samples 64 windows,
    unrolls 8 network steps with checkpoints, back-propagates through them
    and takes one Adam step.  Host time (window sampling) included."""
    import torch

    from paper_2403_12820_gb300.train import Dataset, Trainer

    t0 = time.perf_counter()
    data = Dataset(count=512, n=64, steps=200, device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    tr = Trainer(data, batch=64, unroll=8, device=dev)
    losses = [tr.step() for _ in range(3)]
    torch.cuda.synchronize()
    iters = max(1, args.train_iters)
    t0 = time.perf_counter()
    for _ in range(iters):
        losses.append(tr.step())
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    win = 64 * 8 * data.nodes
    out = {"workload": "train: 512 trajectories of 64 x 64 x 200 plain steps (seed 1004); batch 64 windows, "
                       "8-step unroll, Adam lr 1e-3, FP32",
           "iters_per_s": iters / el, "windows_per_s": 64 * iters / el,
           "unrolled_node_steps_per_s": win * iters / el, "iters": iters,
           "dataset_generation_s": gen_s, "loss_first": losses[0], "loss_last": losses[-1]}
    # the same iterations with the literal cell (39 trainable weights)
    tp = Trainer(data, batch=64, unroll=8, device=dev, cell="pcell")
    lp = [tp.step() for _ in range(3)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(iters):
        lp.append(tp.step())
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    out["pcell"] = {"iters_per_s": iters / el, "unrolled_node_steps_per_s": win * iters / el,
                    "loss_first": lp[0], "loss_last": lp[-1]}
    # the differential-evolution pre-process (Sec. 3.2.1, Table 1): 36
    # members x 6 group scales; every member is one loss-only Eq. 8 call on
    # one batch of 64 windows
    from paper_2403_12820_gb300 import workloads as wl
    out["de_preprocess"] = {}
    for cell, gens in (("pcell", args.de_generations), ("cnn", max(1, args.de_generations // 2))):
        td = Trainer(data, batch=64, unroll=8, device=dev, cell=cell)
        res = td.pre_process(wl.de_draws(seed=2007, pop=36, dim=6, generations=gens))
        out["de_preprocess"][cell] = {
            "population": 36, "generations": gens, "evals": res["evals"], "seconds": res["seconds"],
            "evals_per_s": res["evals"] / res["seconds"],
            "unrolled_node_steps_per_s": res["evals"] * win / res["seconds"],
            "loss_unscaled": float(res["initial_fitness"][0]), "loss_best": res["f"],
            "scales": [round(float(v), 4) for v in res["x"]]}
    return out


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        out = run_reference(args, rank, int(os.environ.get("WORLD_SIZE", "1")))
        if out is not None:
            print(json.dumps(out), flush=True)
        return 0
    if args.only is not None:
        import torch
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        fn = {"cnn": lambda: run_cnn(args, dev), "cnn_step": lambda: run_cnn_step(args, dev),
              "mixed": lambda: run_mixed(args, dev),
              "pcell": lambda: run_pcell(args, dev, None),
              "larger_step": lambda: run_larger_step(args, dev, None),
              "train": lambda: run_train(args, dev), "single_cloth": lambda: run_single_cloth(dev)}[args.only]
        print(json.dumps({"section": args.only, "result": fn()}), flush=True)
        return 0
    rank, world, local = dist_setup(args.gpus)
    out = run_plain(args, rank, world, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
