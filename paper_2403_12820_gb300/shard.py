"""Splitting the work over GPUs (one process per GPU, torch.distributed).

Cloths are independent (Sec. 3.1: forces act along springs inside one
cloth), so a batch is split by whole cloths and the ranks exchange nothing
while they step: `partition` assigns the cloths largest first, each to the
rank with the fewest nodes so far.  Training is data parallel: every rank
evaluates the Eq. 8 loss on its own windows and the gradients are averaged
with one all-reduce before the identical Adam step on every rank
(`average_gradient`).
"""
from __future__ import annotations


def partition(sizes, world: int) -> list[list[int]]:
    """Indices of the cloths (node counts `sizes`) for each of `world` ranks:
    largest first, each to the rank with the smallest load so far (ties to
    the lowest rank).  The loads then differ by at most the largest cloth.
    Each rank's list is in ascending index order."""
    if world < 1:
        raise ValueError("world must be at least 1")
    sizes = [int(s) for s in sizes]
    if any(s < 0 for s in sizes):
        raise ValueError("sizes must be non-negative")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def take(cfg: dict, idx: list[int]) -> dict:
    """The sub-batch of a workload dict (specs, pins, x, v) at `idx`."""
    out = dict(cfg)
    for k in ("specs", "pins", "x", "v"):
        out[k] = [cfg[k][i] for i in idx]
    return out


def average_gradient(grad, count: float, group=None):
    """Turn this rank's gradient of a mean loss over `count` terms into the
    gradient of the mean over every rank's terms, in place: one all-reduce
    of count * grad and of count, then a division.  With one process (or no
    process group) the gradient is left as it is.  `grad` lives where the
    group's backend wants it (CUDA for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return grad
    c = torch.tensor([float(count)], dtype=torch.float64, device=grad.device)
    grad.mul_(float(count))
    dist.all_reduce(grad, group=group)
    dist.all_reduce(c, group=group)
    grad.div_(float(c.item()))
    return grad
