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
