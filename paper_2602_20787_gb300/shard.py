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

Rank loss is detected on the host, between steps. A Heartbeat posts each step
to a key-value store before the step's launches. A rank that crashed, hung or
left posts nothing more, so the others raise RankLost before their next launch
instead of entering a collective that would never complete. A process group
created with a short timeout is the second line: a collective whose peer died
ends with an error.
"""
from __future__ import annotations

import time

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


class RankLost(RuntimeError):
    """A peer did not reach a step: `ranks` are the ranks that failed to post
    `step` (crashed, hung or left)."""

    def __init__(self, ranks, step: int):
        super().__init__(f"rank(s) {list(ranks)} did not reach step {step}")
        self.ranks = list(ranks)
        self.step = int(step)


class Heartbeat:
    """Liveness of the ranks between steps, through a key-value store: a
    torch.distributed store, or anything with set(key, value) and
    check([key]) -> bool.

    beat(step) posts this rank's step. It returns once every rank has posted
    the same step. It raises RankLost naming the ranks that did not post it
    within `timeout` seconds; a rank that called leave() is named at once. Call
    beat before a step's launches, so that no kernel or collective is in flight
    when a loss is found."""

    def __init__(self, store, rank: int, world: int, timeout: float = 2.0, poll: float = 0.005,
                 prefix: str = "heartbeat"):
        if world < 1 or not (0 <= rank < world) or not timeout > 0:
            raise ValueError("need 0 <= rank < world and timeout > 0")
        self.store, self.rank, self.world = store, rank, world
        self.timeout, self.poll, self.prefix = float(timeout), float(poll), prefix

    def _key(self, step: int, r: int) -> str:
        return f"{self.prefix}/step/{step}/{r}"

    def _left(self, r: int) -> str:
        return f"{self.prefix}/left/{r}"

    def beat(self, step: int) -> None:
        self.store.set(self._key(step, self.rank), b"1")
        deadline = time.monotonic() + self.timeout
        pending = [r for r in range(self.world) if r != self.rank]
        while True:
            pending = [r for r in pending if not self.store.check([self._key(step, r)])]
            if not pending:
                break
            left = [r for r in pending if self.store.check([self._left(r)])]
            if left:
                raise RankLost(left, step)
            if time.monotonic() >= deadline:
                raise RankLost(pending, step)
            time.sleep(self.poll)
        # every rank has posted `step`, so none still waits on this rank's previous key
        delete = getattr(self.store, "delete_key", None)
        if delete is not None and step > 0:
            delete(self._key(step - 1, self.rank))

    def leave(self, step: int) -> None:
        """Announce that this rank stops after `step` (call it between steps)."""
        self.store.set(self._left(self.rank), str(int(step)).encode())
