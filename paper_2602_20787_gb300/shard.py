"""Row sharding of the direct S1xR2 force across ranks (host-side logic).

The i-rows of the pair sum are independent (each particle's acceleration sums
over every j), so the force work splits into contiguous ranges of i with no
reduction between ranks. The only exchange a sharded force evaluation needs is
one all-gather of the positions, after which every rank holds the full j-set and
computes its own rows; the KDK kick and drift are local to each rank's rows, and
the conserved quantities need one all-reduce of a few sums.

Each rank's rows are evaluated with the same per-i sum order as on one rank, so
the sharded result equals the unsharded one bit for bit. This module holds the
partition, the exchange and the rank reductions; they run with any
torch.distributed backend (NCCL between GPUs, gloo on the host).
"""
from __future__ import annotations

import numpy as np


def partition(n: int, world: int):
    """Balanced contiguous row ranges [(i0, i1)] for world ranks (sizes differ by <= 1)."""
    if n < 0 or world < 1:
        raise ValueError("need n >= 0 and world >= 1")
    base, extra = divmod(n, world)
    out, i0 = [], 0
    for r in range(world):
        i1 = i0 + base + (1 if r < extra else 0)
        out.append((i0, i1))
        i0 = i1
    return out


def gather_rows(local, n: int, group=None):
    """All-gather of each rank's rows (tensor (k_r, c), contiguous ranges in rank
    order, sizes from partition(n, world)) into the full (n, c) array on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    ranges = partition(n, world)
    width = max(i1 - i0 for i0, i1 in ranges)
    c = local.shape[1]
    pad = torch.zeros((width, c), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[: i1 - i0] for p, (i0, i1) in zip(parts, ranges)], 0)


def max_over_ranks(value: float, group=None, device=None) -> float:
    """Maximum of a per-rank scalar (the timing rule of the benchmark)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(values, group=None, device=None) -> np.ndarray:
    """Element-wise sum of per-rank vectors (conserved quantities of the shards)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(values, dtype=np.float64), device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()
