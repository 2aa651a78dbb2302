"""Row sharding of the direct S1xR2 force across ranks (host-side logic).

The i-rows of the pair sum are independent (each particle's acceleration sums
over every j), so the force work splits into contiguous ranges of i with no
reduction between ranks. The only exchange a sharded force evaluation needs is
one all-gather of the positions, after which every rank holds the full j-set and
computes its own rows; the KDK kick and drift are local to each rank's rows, and
the conserved quantities need one all-reduce of a few sums.

This module holds the partition, the exchange and the rank reductions, and
ShardedSimulation, which drives one cylinder's KDK steps across the ranks with
one all-gather per step; they run with any torch.distributed backend (NCCL
between GPUs, gloo on the host). The rank's compute is pluggable: GpuRows runs
it through the C ABI (steps_cyl_shard, steps_cyl_shard_drift and
steps_cyl_shard_kick); a backend whose per-row sums keep the unsharded order
reproduces the unsharded run bit for bit.

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


def all_gather_rows(send, group=None):
    """All-gather of equal-sized per-rank tensors (chunk, c) into (world * chunk, c)
    in rank order: NCCL's gather into one tensor for CUDA tensors, the list form
    otherwise (gloo)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if send.is_cuda:
        out = torch.empty((world * send.shape[0],) + tuple(send.shape[1:]), dtype=send.dtype, device=send.device)
        dist.all_gather_into_tensor(out, send.contiguous(), group=group)
        return out
    parts = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(parts, send.contiguous(), group=group)
    return torch.cat(parts, 0)


def reduce_scatter_rows(sums, group=None):
    """Sum over the ranks of a rank-major tensor (world * k, ...) and hand rank r
    its slice r of k rows: NCCL's reduce-scatter for CUDA tensors, an all-reduce
    and a slice otherwise (gloo has no reduce-scatter). Integer tensors sum
    exactly, so the result does not depend on the order of the ranks."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    k = sums.shape[0] // world
    if sums.is_cuda:
        import torch
        out = torch.empty((k,) + tuple(sums.shape[1:]), dtype=sums.dtype, device=sums.device)
        dist.reduce_scatter_tensor(out, sums.contiguous(), op=dist.ReduceOp.SUM, group=group)
        return out
    tot = sums.clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM, group=group)
    return tot[rank * k:(rank + 1) * k].contiguous()


class GpuRows:
    """A rank's rows on its GPU: a steps_cyl context made from the full state
    (the same on every rank) and then sharded with steps_cyl_shard. Train or
    install a modelled tail on the context before handing it over.

    drift(dt) runs steps_cyl_shard_drift and returns the send buffer (chunk, 8)
    float32. Then either kick(recv) runs steps_cyl_shard_kick on the gathered
    rows (the row step), or, when `symmetric` is set, force(recv) returns the
    rank's pair sums (steps_cyl_shard_force) and finish(own) completes the step
    from the reduce-scattered sums of its rows (steps_cyl_shard_finish). The
    context's stream must be the current torch stream, so that the collectives
    between the calls are ordered after the one before and before the next."""

    def __init__(self, sim, rank: int, world: int, symmetric: bool = True):
        import torch
        from . import steps_cyl as sc
        self.sc, self.sim, self.rank, self.world = sc, sim, rank, world
        self.k0, self.k1, self.chunk = sc.steps_cyl_shard(sim.ctx, rank, world)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.send = torch.zeros((self.chunk, 8), dtype=torch.float32, device=self.device)
        avail, sums_len = sc.steps_cyl_shard_mode(sim.ctx)
        self.symmetric = bool(symmetric and avail)
        self.pair_sums = torch.zeros(sums_len, dtype=torch.int64, device=self.device) if self.symmetric else None

    def drift(self, dt: float):
        self.sc.steps_cyl_shard_drift(self.sim.ctx, dt, self.send)
        return self.send

    def kick(self, recv):
        self.sc.steps_cyl_shard_kick(self.sim.ctx, recv)

    def force(self, recv):
        self.sc.steps_cyl_shard_force(self.sim.ctx, recv, self.pair_sums)
        return self.pair_sums

    def finish(self, own):
        self.sc.steps_cyl_shard_finish(self.sim.ctx, own)

    def sums(self):
        """(P[3], L_z, kinetic energy, mass) of the owned rows, and (a, t)."""
        d = self.sim.diagnostics()
        return np.array([d[0], d[1], d[2], d[3], d[4], d[7]]), (float(d[5]), float(d[6]))

    def state(self):
        """Positions and velocities in caller order, zeros outside the owned rows."""
        x, v, _, _ = self.sim.state()
        return np.concatenate([x, v], 1)

    def check(self, tail: int, particles: int = 1024):
        """(median, p99.9) of the modelled tail's error on a sample of the owned rows."""
        rep = self.sc.steps_cyl_check_tail(self.sim.ctx, tail, particles)
        return float(rep[0]), float(rep[1])

    def set_tail(self, tail: int):
        self.sc.steps_cyl_set_tail(self.sim.ctx, tail)


class ShardedSimulation:
    """One cylinder whose rows are split across the ranks of a process group
    (Sect. 2.4's distributed direct engine, one rank per GPU). Each KDK step is
    compute.drift(dt) on the rank's rows and one all-gather of the packed rows
    of every rank. Then, in the row step, compute.kick(gathered): the pair force
    of the rank's rows against every particle, the background and the second
    kick, with no other exchange. In the symmetric step (compute.symmetric),
    compute.force(gathered) evaluates the rank's share of the unordered pairs
    for both particles of each, one reduce-scatter sums them onto the ranks
    that own the rows, and compute.finish(own) completes the step. `compute` is the rank's backend (GpuRows, or any
    object with the same drift / kick (or force / finish) / sums / state / check
    / set_tail methods and a `device` attribute for the collectives' tensors).

    With a modelled tail (tail = STEPS_TAIL_SURROGATE or STEPS_TAIL_TABLE) and
    check_every > 0, every check_every steps each rank checks a sample of its
    rows against the plain image sum; the largest median and p99.9 over the
    ranks decide, and a failed check switches every rank to the plain sum
    together (returned by step() as False)."""

    def __init__(self, compute, group=None, tail: int = 0, check_every: int = 0, bounds=(1e-5, 1e-3),
                 check_particles: int = 1024):
        self.compute, self.group = compute, group
        self.tail, self.check_every, self.bounds = int(tail), int(check_every), bounds
        self.check_particles = int(check_particles)
        self.steps = 0
        self.last_check = None

    def step(self, dt: float, nsteps: int = 1) -> bool:
        ok = True
        for _ in range(nsteps):
            send = self.compute.drift(dt)
            recv = all_gather_rows(send, self.group)
            if getattr(self.compute, "symmetric", False):
                # each unordered pair once across the ranks, then the sums of every
                # rank's rows gathered to it (integer sums: exact in any order)
                self.compute.finish(reduce_scatter_rows(self.compute.force(recv), self.group))
            else:
                self.compute.kick(recv)
            self.steps += 1
            if self.tail and self.check_every > 0 and self.steps % self.check_every == 0:
                ok = self._check() and ok
        return ok

    def _check(self) -> bool:
        import torch
        import torch.distributed as dist
        med, p999 = self.compute.check(self.tail, self.check_particles)
        t = torch.tensor([med, p999], dtype=torch.float64, device=getattr(self.compute, "device", None))
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=self.group)
        med, p999 = float(t[0]), float(t[1])
        self.last_check = (med, p999)
        if med <= self.bounds[0] and p999 <= self.bounds[1]:
            return True
        self.tail = 0
        self.compute.set_tail(0)
        return False

    def diagnostics(self) -> np.ndarray:
        """P[3], L_z, kinetic energy, mass of the whole cylinder, then a and t."""
        sums, (a, t) = self.compute.sums()
        tot = sum_over_ranks(sums, group=self.group, device=getattr(self.compute, "device", None))
        return np.concatenate([tot, [a, t]])

    def state(self) -> np.ndarray:
        """(n, 6) positions and velocities of every particle in caller order,
        assembled from the ranks' rows (every rank receives it)."""
        import torch
        import torch.distributed as dist
        own = self.compute.state()
        t = torch.tensor(own, dtype=torch.float64, device=getattr(self.compute, "device", None))
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
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
