"""Row sharding across ranks, emulated with two gloo ranks on the host: the
partition, the position all-gather, and the max-over-ranks timing rule. The
sharded pair field (each rank its rows against the gathered positions, here
with the FP64 oracle) equals the unsharded one bit for bit."""
import os
import socket

import numpy as np
import pytest

from paper_2602_20787_gb300 import shard


def test_partition_is_balanced_and_complete():
    for n, world in ((97, 2), (10, 3), (5, 8), (0, 2), (1 << 16, 7)):
        parts = shard.partition(n, world)
        assert len(parts) == world and parts[0][0] == 0 and parts[-1][1] == n
        sizes = [b - a for a, b in parts]
        assert max(sizes) - min(sizes) <= 1
        assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
    with pytest.raises(ValueError):
        shard.partition(4, 0)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2602_20787_gb300 import ics
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, n_cut = 97, 5
        d = ics.particle_load(n, 31, 1.0)           # every rank draws the same seeded load
        i0, i1 = shard.partition(n, world)[rank]
        local = torch.tensor(d["pos"][i0:i1])
        full = shard.gather_rows(local, n).numpy()
        assert np.array_equal(full, d["pos"])
        g_local = oracle.pair_field(full, d["m"], d["h"], 1.0, 1.0, n_cut, idx=np.arange(i0, i1))
        g = shard.gather_rows(torch.tensor(g_local), n).numpy()
        tmax = shard.max_over_ranks(1.5 + rank)
        mass = shard.sum_over_ranks([d["m"][i0:i1].sum(), float(i1 - i0)])
        if rank == 0:
            np.save(os.path.join(out_dir, "g.npy"), g)
            np.save(os.path.join(out_dir, "misc.npy"), np.array([tmax, mass[0], mass[1]]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_unsharded_field(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    from paper_2602_20787_gb300 import ics
    oracle.build()
    mp.start_processes(worker, args=(2, free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    g = np.load(tmp_path / "g.npy")
    misc = np.load(tmp_path / "misc.npy")
    d = ics.particle_load(97, 31, 1.0)
    ref = oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, 5)
    np.testing.assert_array_equal(g, ref)
    assert misc[0] == 2.5
    assert misc[1] == pytest.approx(1.0, rel=1e-14) and misc[2] == 97


class OracleRows:
    """A rank's rows computed by the FP64 oracle (test backend of
    ShardedSimulation): the rank holds every particle's position, updated from
    the all-gather each step, and the momenta and field of its own rows. Every
    operation is the oracle KDK's, element by element in the same order (p +=
    g K1, x += p D, z wrapped, then the pair field of its rows against all j
    plus the background), so the sharded run equals the unsharded one bit for
    bit."""

    def __init__(self, pos, p, m, h, n_cut, rho0, cosmo, a, t, rank, world):
        import torch
        import oracle
        from paper_2602_20787_gb300 import ics
        self.orc, self.R = oracle, ics.R_SIM
        self.x, self.p = pos.copy(), p.copy()
        self.m, self.h, self.n_cut, self.rho0, self.c = m, h, n_cut, rho0, cosmo
        self.a, self.t = a, t
        self.n = pos.shape[0]
        parts = shard.partition(self.n, world)
        self.k0, self.k1 = parts[rank]
        self.chunk = max(b - a_ for a_, b in parts)
        self.parts = parts
        self.device = torch.device("cpu")
        self.own = np.arange(self.k0, self.k1)
        self.g = self.field()

    def field(self):
        g = self.orc.pair_field(self.x, self.m, self.h, 1.0, 1.0, self.n_cut, idx=self.own)
        return g + self.orc.background_field(self.x[self.own], self.R, self.n_cut * 1.0, 1.0, self.rho0, mode=1)

    def drift(self, dt):
        import torch
        K1, D, self.K2, self.an = self.orc.kdk_factors(self.c, self.a, dt)
        self.dt = dt
        o = slice(self.k0, self.k1)
        self.p[o] += self.g * K1
        self.x[o] += self.p[o] * D
        z = self.x[o, 2] - 1.0 * np.floor(self.x[o, 2] / 1.0)
        self.x[o, 2] = np.where(z >= 1.0, z - 1.0, z)
        send = np.zeros((self.chunk, 3))
        send[: self.k1 - self.k0] = self.x[o]
        return torch.tensor(send)

    def kick(self, recv):
        r = recv.numpy()
        for q, (a_, b) in enumerate(self.parts):
            self.x[a_:b] = r[q * self.chunk: q * self.chunk + (b - a_)]
        self.g = self.field()
        self.p[self.k0:self.k1] += self.g * self.K2
        self.a = self.an
        self.t += self.dt

    def sums(self):
        d = self.orc.diagnostics(self.x[self.own], self.p[self.own], self.m[self.own], self.a)
        return d, (self.a, self.t)

    def state(self):
        out = np.zeros((self.n, 6))
        out[self.own, :3] = self.x[self.own]
        out[self.own, 3:] = self.p[self.own] / self.a ** 2
        return out


def sharded_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle
    from paper_2602_20787_gb300 import ics
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = ics.WORKLOADS["lcdm_n65536"]
        n, n_cut, steps = 131, 4, 5
        d = ics.particle_load(n, 33, w.M_tot, displaced=True, rho_bar=w.rho_bar)
        p0 = np.random.default_rng(8).normal(0.0, 0.05, (n, 3)) * w.a_start ** 2
        t0, dt = ics.run_schedule(w)
        rows = OracleRows(d["pos"], p0, d["m"], d["h"], n_cut, w.rho_bar, oracle.make_cosmo(), w.a_start, t0,
                          rank, world)
        sim = shard.ShardedSimulation(rows)
        sim.step(20 * dt, steps)
        st = sim.state()
        diag = sim.diagnostics()
        if rank == 0:
            np.save(os.path.join(out_dir, f"state{world}.npy"), st)
            np.save(os.path.join(out_dir, f"diag{world}.npy"), diag)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_simulation_reproduces_the_unsharded_oracle_kdk(tmp_path, world):
    # ShardedSimulation's orchestration (drift, one all-gather, kick per step)
    # with an FP64 oracle compute on gloo ranks against the oracle's own
    # unsharded KDK: positions and momenta bit for bit, diagnostics to rounding
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    from paper_2602_20787_gb300 import ics
    oracle.build()
    mp.start_processes(sharded_worker, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    st = np.load(tmp_path / f"state{world}.npy")
    diag = np.load(tmp_path / f"diag{world}.npy")
    w = ics.WORKLOADS["lcdm_n65536"]
    n, n_cut, steps = 131, 4, 5
    d = ics.particle_load(n, 33, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    p0 = np.random.default_rng(8).normal(0.0, 0.05, (n, 3)) * w.a_start ** 2
    t0, dt = ics.run_schedule(w)
    x, p, a, t = oracle.kdk(d["pos"], p0, d["m"], d["h"], 1.0, 1.0, n_cut, ics.R_SIM, w.rho_bar, 1,
                            oracle.make_cosmo(), w.a_start, t0, 20 * dt, steps)
    np.testing.assert_array_equal(st[:, :3], x)
    np.testing.assert_array_equal(st[:, 3:], p / a ** 2)
    ref = oracle.diagnostics(x, p, d["m"], a)
    scale = np.sum(d["m"][:, None] * np.abs(p))
    np.testing.assert_allclose(diag[:3], ref[:3], rtol=0, atol=1e-14 * scale)
    assert diag[4] == pytest.approx(ref[4], rel=1e-13) and diag[5] == pytest.approx(ref[5], rel=1e-14)
    assert diag[6] == a and diag[7] == t


class OracleSymRows(OracleRows):
    """The symmetric step with an FP64 oracle compute (test backend): force()
    evaluates this rank's 1/world share of the unordered pairs (i < j, in
    lexicographic order) with the oracle's windowed image sum of eq.
    ForceCylindrical, adding m_j f to i and -m_i f to j in a rank-major buffer
    [world][3][chunk]; finish() takes the rank's reduce-scattered rows."""

    symmetric = True

    def force(self, recv):
        import torch
        r = recv.numpy()
        for q, (a_, b) in enumerate(self.parts):
            self.x[a_:b] = r[q * self.chunk: q * self.chunk + (b - a_)]
        world = len(self.parts)
        rank = self.parts.index((self.k0, self.k1))
        iu, ju = np.triu_indices(self.n, 1)
        lo, hi = rank * iu.size // world, (rank + 1) * iu.size // world
        sums = np.zeros((world, 3, self.chunk))
        owner = np.zeros(self.n, dtype=np.int64)
        for q, (a_, b) in enumerate(self.parts):
            owner[a_:b] = q
        first = np.array([a_ for a_, _ in self.parts])
        for i, j in zip(iu[lo:hi], ju[lo:hi]):
            f, _ = self.orc.image_force(self.x[i] - self.x[j], self.h[i] + self.h[j], 1.0, self.n_cut)
            sums[owner[i], :, i - first[owner[i]]] += self.m[j] * f
            sums[owner[j], :, j - first[owner[j]]] -= self.m[i] * f
        return torch.tensor(sums.reshape(world * 3, self.chunk))

    def finish(self, own):
        g = own.numpy().reshape(3, self.chunk)[:, : self.k1 - self.k0].T.copy()
        self.g = g + self.orc.background_field(self.x[self.own], self.R, self.n_cut * 1.0, 1.0, self.rho0, mode=1)
        self.p[self.k0:self.k1] += self.g * self.K2
        self.a = self.an
        self.t += self.dt


def sym_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle
    from paper_2602_20787_gb300 import ics
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = ics.WORKLOADS["lcdm_n65536"]
        n, n_cut, steps = 131, 4, 3
        d = ics.particle_load(n, 34, w.M_tot, displaced=True, rho_bar=w.rho_bar)
        p0 = np.random.default_rng(9).normal(0.0, 0.05, (n, 3)) * w.a_start ** 2
        t0, dt = ics.run_schedule(w)
        rows = OracleSymRows(d["pos"], p0, d["m"], d["h"], n_cut, w.rho_bar, oracle.make_cosmo(), w.a_start, t0,
                             rank, world)
        sim = shard.ShardedSimulation(rows)
        sim.step(20 * dt, steps)
        st = sim.state()
        if rank == 0:
            np.save(os.path.join(out_dir, f"symstate{world}.npy"), st)
    finally:
        dist.destroy_process_group()


def test_symmetric_sharded_step_matches_the_oracle_kdk(tmp_path):
    # the symmetric step's orchestration: drift, all-gather, each rank's share
    # of the unordered pairs for both particles, reduce-scatter, finish; against
    # the oracle's unsharded KDK (the pair sums are added in another order, so
    # to FP64 rounding, not bit for bit)
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    from paper_2602_20787_gb300 import ics
    oracle.build()
    world = 3
    mp.start_processes(sym_worker, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    st = np.load(tmp_path / f"symstate{world}.npy")
    w = ics.WORKLOADS["lcdm_n65536"]
    n, n_cut, steps = 131, 4, 3
    d = ics.particle_load(n, 34, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    p0 = np.random.default_rng(9).normal(0.0, 0.05, (n, 3)) * w.a_start ** 2
    t0, dt = ics.run_schedule(w)
    x, p, a, _ = oracle.kdk(d["pos"], p0, d["m"], d["h"], 1.0, 1.0, n_cut, ics.R_SIM, w.rho_bar, 1,
                            oracle.make_cosmo(), w.a_start, t0, 20 * dt, steps)
    disp = np.abs(x - d["pos"]).max()
    np.testing.assert_allclose(st[:, :3], x, rtol=0, atol=1e-12 * disp)
    v = p / a ** 2
    np.testing.assert_allclose(st[:, 3:], v, rtol=0, atol=1e-12 * np.abs(v).max())
