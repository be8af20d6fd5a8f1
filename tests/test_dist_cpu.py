"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Cloths are independent, so ranks share no data; the only communication is
the barrier around the timed region and the max over ranks of its length.
These run without a GPU: two spawned processes rendezvous on 127.0.0.1.
"""
import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    r, w, local = bench.dist_setup(world)
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    # each rank's timed region differs; every rank must see the slowest
    m = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    # whole-job rate = all ranks' node-steps / the slowest rank's time
    nodes, steps = 1000 * (rank + 1), 10
    rate = w * 1000 * steps / (bench.max_over_ranks(2.0 * (rank + 1), w))
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{m} {rate} {nodes}\n")
    import torch.distributed as dist
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_barrier_and_max(tmp_path):
    port = _free_port()
    tmp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    vals = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(2)]
    for v in vals:
        assert float(v[0]) == 15.0              # max over ranks, seen by both
        assert float(v[1]) == 2 * 1000 * 10 / 4.0


def _ref_main(rank: int, world: int, port: int, out_dir: str):
    """`--impl reference` under torchrun: rank 0 alone prints; others exit."""
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    args = bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    if rank != 0:
        out = bench.run_reference(args, rank, world)
        with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as fh:
            fh.write(repr(out))


def test_reference_arm_other_ranks_do_no_work(tmp_path):
    _ref_main(1, 2, _free_port(), str(tmp_path))
    assert open(tmp_path / "ref1.txt").read() == "None"


def test_reference_arm_line_keeps_the_contract():
    """Rank 0 of `--impl reference` times the FP64 oracle on the host cores
    and returns the contract's JSON line: the plain arm's metric and unit,
    the requested steps and warm-up, and cpu_baseline / e2e describing the
    same run."""
    import bench
    args = bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    out = bench.run_reference(args, 0, 1)
    assert out["impl"] == "reference"
    assert out["metric"].startswith("cloth node-steps/s") and out["unit"] == "node-steps/s"
    assert out["value"] > 0 and out["higher_is_better"] is True and out["vs_baseline"] is None
    assert out["steps"] == 1 and out["warmup"] == 3 and out["n_gpus"] == 1 and out["scaling"] == "weak"
    assert out["ms_per_step"] > 0 and out["dtype"] == "f64" and out["data"] == "synthetic"
    assert out["config"]["workload"].startswith("plain_batch")
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


# ------------------------------------------------------------------ the split
def test_partition_covers_the_batch_and_balances_within_the_largest_cloth():
    """Largest first, each cloth to the least-loaded rank: the shards are
    disjoint, their union is the batch, and the loads differ by at most the
    largest cloth (checked on the 64-cloth batch's node counts and random
    ones, for 1 to 8 ranks)."""
    import numpy as np

    from paper_2403_12820_gb300 import shard
    from paper_2403_12820_gb300 import workloads as wl
    cfg = wl.plain_batch()
    sets = [[s["rows"] * s["cols"] for s in cfg["specs"]]]
    rng = np.random.default_rng(5)
    sets += [list(rng.integers(1, 10 ** 6, size=k)) for k in (1, 3, 17, 200)]
    for sizes in sets:
        for world in range(1, 9):
            parts = shard.partition(sizes, world)
            assert len(parts) == world
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(len(sizes)))
            loads = [sum(sizes[i] for i in p) for p in parts]
            assert max(loads) - min(loads) <= max(sizes)
    # exact small case: 7, 5, 4, 3 over 2 ranks -> {7, 3} and {5, 4}
    assert shard.partition([3, 7, 4, 5], 2) == [[0, 1], [2, 3]]


def _grad_main(rank: int, world: int, port: int, out_dir: str):
    """Each rank: the mean over its windows of per-window gradients (the
    oracle's Eq. 8 gradients stand in for the GPU's), averaged over the ranks
    by shard.average_gradient."""
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2403_12820_gb300 import shard
    dist.init_process_group("gloo")
    g_all = np.load(os.path.join(out_dir, "g.npy"))
    mine = [0, 1, 2] if rank == 0 else [3, 4]          # uneven shards
    g = torch.from_numpy(g_all[mine].mean(axis=0))
    shard.average_gradient(g, len(mine))
    np.save(os.path.join(out_dir, f"avg{rank}.npy"), g.numpy())
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_data_parallel_gradient_equals_the_single_rank_gradient(tmp_path):
    """Two gloo ranks with 3 and 2 windows: the averaged gradient equals the
    gradient of the mean loss over all 5 windows on one rank, to 1e-6."""
    import numpy as np

    import oracle
    from paper_2403_12820_gb300 import workloads as wl
    rng = np.random.default_rng(71)
    w = wl.kaiming_blob(72, in_scale=(50.0,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3, bias_sigma=0.1)
    grads = []
    for k in range(5):
        sp = wl.cloth_spec(6, 7, p=rng.normal(0, 0.5))
        x0, v0 = wl.sag_state(sp, rng, amp=0.01, vamp=0.05)
        pins = [0, 6]
        tg, xt, vt = [], x0.astype(np.float64), v0.astype(np.float64)
        for _ in range(2):
            xt, vt = oracle.step(sp, xt, vt, pins=pins, steps=1)
            tg.append(xt)
        a_true = (oracle.total_force(sp, x0, v0) - oracle.pressure_force(sp, x0)) / sp["m"]
        _, g = oracle.unroll_loss(w.astype(np.float64), sp, pins, x0, v0, np.array(tg), a_true, 0.5, 9.81, sp["h"])
        grads.append(g)
    g_all = np.array(grads)
    np.save(tmp_path / "g.npy", g_all)
    tmp.spawn(_grad_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    ref = g_all.mean(axis=0)
    for r in range(2):
        got = np.load(tmp_path / f"avg{r}.npy")
        assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


def test_average_gradient_without_a_process_group_is_the_identity():
    import torch

    from paper_2403_12820_gb300 import shard
    g = torch.arange(5, dtype=torch.float32)
    assert torch.equal(shard.average_gradient(g.clone(), 3), g)
