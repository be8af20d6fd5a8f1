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
