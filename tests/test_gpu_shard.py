"""GPU parity of the row-sharded path (steps_cyl_shard, steps_cyl_shard_drift,
steps_cyl_shard_kick; Sect. 2.4's distributed direct engine) through the C ABI.

Every run here has one GPU, so several ranks are emulated in one process: each
rank is its own context on the same stream, their launches are independent (no
kernel waits on another), and the all-gather between the two halves of a step
is a device copy in rank order (and the reduce-scatter of the symmetric step an
integer sum of the ranks' buffers, sliced by rank). One rank alone must
reproduce the unsharded KDK bit for bit; two and three ranks, in the row step
and in the symmetric step, must match the FP64 oracle's KDK to the FP32
tolerance, and the unsharded FP32 forms to their rounding."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20787_gb300 import shard, steps_cyl
    steps_cyl.load()
    return torch, steps_cyl, shard


def load(n=1000, seed=51):
    w = ics.WORKLOADS["lcdm_n65536"]
    d = ics.particle_load(n, seed, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    d["vel"] = np.random.default_rng(seed).normal(0.0, 0.05, (n, 3))
    t0, dt = ics.run_schedule(w)
    return w, d, t0, dt


def config(sc, w, t0, precision, stream, **kw):
    return sc.Config(n_cut=w.n_cut, precision=precision, comoving=True, a_start=w.a_start, t_start=t0,
                     rho_bar=w.rho_bar, reorder_every=-1, stream=stream, **kw)


def emulated_ranks(torch, sc, shard, cfg, d, world, symmetric=False):
    sims = [sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"]) for _ in range(world)]
    return [shard.GpuRows(s, r, world, symmetric=symmetric) for r, s in enumerate(sims)]


def step_emulated(torch, ranks, dt, steps):
    for _ in range(steps):
        sends = [r.drift(dt) for r in ranks]
        recv = torch.cat(sends, 0)            # the all-gather, in rank order
        if ranks[0].symmetric:
            sums = [r.force(recv) for r in ranks]
            tot = torch.stack(sums, 0).sum(0)  # the reduce-scatter: integer sums over the ranks ...
            k = tot.shape[0] // len(ranks)
            for q, r in enumerate(ranks):     # ... and rank q's slice
                r.finish(tot[q * k:(q + 1) * k].contiguous())
        else:
            for r in ranks:
                r.kick(recv)


def assembled_state(ranks):
    st = sum(r.state() for r in ranks)        # each rank: its rows, zeros elsewhere
    return st[:, :3], st[:, 3:]


def test_one_rank_is_the_unsharded_kdk_bit_for_bit(env):
    torch, sc, shard = env
    w, d, t0, dt = load()
    stream = torch.cuda.current_stream().cuda_stream
    cfg = config(sc, w, t0, sc.STEPS_FP32_KAHAN, stream)
    ref = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    ref.step(dt, 5)
    x_ref, v_ref, a_ref, t_ref = ref.state()
    ref.close()
    (rows,) = emulated_ranks(torch, sc, shard, cfg, d, 1)
    assert (rows.k0, rows.k1, rows.chunk) == (0, 1000, 1000)
    step_emulated(torch, [rows], dt, 5)
    x, v, a, t = rows.sim.state()
    np.testing.assert_array_equal(x, x_ref)
    np.testing.assert_array_equal(v, v_ref)
    assert a == a_ref and t == t_ref
    rows.sim.close()


@pytest.mark.parametrize("world,symmetric", [(2, False), (3, False), (2, True), (3, True)])
def test_emulated_ranks_match_the_oracle_kdk(env, world, symmetric):
    # FP32-Kahan sharded steps (the row step, and the symmetric step with its
    # reduce-scatter) against the FP64 oracle's KDK, at the FP32 tolerance of
    # the unsharded KDK parity test (1e-5 of the motion)
    torch, sc, shard = env
    w, d, t0, dt = load()
    steps = 4
    stream = torch.cuda.current_stream().cuda_stream
    ranks = emulated_ranks(torch, sc, shard, config(sc, w, t0, sc.STEPS_FP32_KAHAN, stream), d, world, symmetric)
    assert all(r.symmetric == symmetric for r in ranks)
    # 1000 rows are 8 blocks of 128: balanced contiguous block ranges
    assert ranks[0].k0 == 0 and ranks[-1].k1 == 1000
    assert all(ranks[r].k1 == ranks[r + 1].k0 for r in range(world - 1))
    assert all(r.k0 % 128 == 0 for r in ranks)
    step_emulated(torch, ranks, dt, steps)
    x, v = assembled_state(ranks)
    xo, po, ao, _ = oracle.kdk(d["pos"], d["vel"] * w.a_start ** 2, d["m"], d["h"], 1.0, 1.0, w.n_cut, ics.R_SIM,
                               w.rho_bar, 1, oracle.make_cosmo(), w.a_start, t0, dt, steps)
    dx = x - xo
    dx[:, 2] = np.mod(dx[:, 2] + 0.5, 1.0) - 0.5
    disp = np.abs(xo - d["pos"])
    disp[:, 2] = np.minimum(disp[:, 2], 1.0 - disp[:, 2])
    assert np.abs(dx).max() <= 1e-5 * disp.max()
    vo = po / ao ** 2
    dv_o = vo - d["vel"] * (w.a_start / ao) ** 2      # the velocity the forces added
    assert np.abs(v - vo).max() <= 1e-5 * np.abs(dv_o).max()
    # the ranks' diagnostics add up to the oracle's sums of its state
    tot = sum(r.sums()[0] for r in ranks)
    ref = oracle.diagnostics(xo, po, d["m"], ao)
    pscale = np.sum(d["m"][:, None] * np.abs(po))
    np.testing.assert_allclose(tot[:3], ref[:3], rtol=0, atol=1e-6 * pscale)
    assert tot[5] == pytest.approx(ref[5], rel=1e-13)
    for r in ranks:
        assert r.sums()[1][0] == pytest.approx(ao, rel=1e-14)
        with pytest.raises(sc.StepsError):
            sc.steps_cyl_set_precision(r.sim.ctx, sc.STEPS_FP64)
        r.sim.close()


def test_emulated_ranks_match_the_unsharded_fp32_forms(env):
    # FP32-Kahan and the learned tail (trained and accepted before sharding):
    # the sharded forces and KDK steps agree with the unsharded context to FP32
    # rounding (the work split of each row differs, the arithmetic does not)
    torch, sc, shard = env
    w = ics.WORKLOADS["surrogate_n65536"]
    n = 3000
    d = ics.particle_load(n, 52, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    t0 = ics.lcdm_time_of_a(w.a_start)
    dt = 0.005 * t0
    stream = torch.cuda.current_stream().cuda_stream
    cfg = sc.Config(n_cut=w.n_cut, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, comoving=True, a_start=w.a_start,
                    t_start=t0, rho_bar=w.rho_bar, reorder_every=-1, stream=stream)
    train = sc.steps_cyl_train_cfg_default()
    sims = [sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"]) for _ in range(3)]
    for s in sims:
        sc.steps_cyl_train_surrogate(s.ctx, train)   # deterministic: the same network on every context
        sc.steps_cyl_set_tail(s.ctx, sc.STEPS_TAIL_SURROGATE)
    np.testing.assert_array_equal(sc.steps_cyl_get_surrogate(sims[0].ctx), sc.steps_cyl_get_surrogate(sims[1].ctx))
    ref, ranks = sims[0], [shard.GpuRows(s, r, 2, symmetric=False) for r, s in enumerate(sims[1:])]
    a_ref = ref.forces()
    a_sh = sum(r.sim.forces() for r in ranks)
    rel = np.linalg.norm(a_sh - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)
    assert np.median(rel) <= 1e-6 and rel.max() <= 1e-4, (np.median(rel), rel.max())
    ref.step(dt, 3)
    step_emulated(torch, ranks, dt, 3)
    x_ref, v_ref, _, _ = ref.state()
    x, v = assembled_state(ranks)
    dx = x - x_ref
    dx[:, 2] = np.mod(dx[:, 2] + 0.5, 1.0) - 0.5
    disp = np.abs(x_ref - d["pos"])
    disp[:, 2] = np.minimum(disp[:, 2], 1.0 - disp[:, 2])
    assert np.abs(dx).max() <= 1e-5 * disp.max()
    assert np.abs(v - v_ref).max() <= 1e-5 * np.abs(v_ref - d["vel"]).max()
    # a check of the owned rows runs against the plain sum
    med, p999 = ranks[0].check(sc.STEPS_TAIL_SURROGATE, 256)
    assert med <= 1e-5 and p999 <= 1e-3
    for s in sims:
        s.close()


def test_symmetric_sharded_step_matches_unsharded_learned_tail(env):
    # the learned tail (trained and accepted before sharding) in the symmetric
    # sharded step: each rank's share of the unordered pairs, the integer sums
    # reduce-scattered; KDK steps agree with the unsharded context to FP32
    # rounding, and the step is deterministic
    torch, sc, shard = env
    w = ics.WORKLOADS["production_n524288"]
    n = 2600
    d = ics.workload_ics(w, n=n)
    t0, dt = ics.run_schedule(w)
    stream = torch.cuda.current_stream().cuda_stream
    cfg = sc.Config(n_cut=w.n_cut, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, comoving=True, a_start=w.a_start,
                    t_start=t0, rho_bar=w.rho_bar, reorder_every=-1, stream=stream)
    runs = []
    for world in (1, 2, 3, 3):
        sims = [sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"]) for _ in range(world)]
        for s in sims:
            sc.steps_cyl_train_surrogate(s.ctx, sc.steps_cyl_train_cfg_default())
            sc.steps_cyl_set_tail(s.ctx, sc.STEPS_TAIL_SURROGATE)
        if world == 1:
            sims[0].step(dt, 4)
            x, v, a, _ = sims[0].state()
            runs.append((x, v, a))
            sims[0].close()
            continue
        ranks = [shard.GpuRows(s, r, world) for r, s in enumerate(sims)]
        assert all(r.symmetric for r in ranks)
        step_emulated(torch, ranks, dt, 4)
        x, v = assembled_state(ranks)
        ev = sc.steps_cyl_last_eval(ranks[0].sim.ctx)
        assert ev["symmetric"] and ev["pairs_evaluated"] < 0.6 * n * n / world
        runs.append((x, v, ranks[0].sums()[1][0]))
        for s in sims:
            s.close()
    x1, v1, a1 = runs[0]
    dv1 = v1 - d["vel"]
    for x, v, a in runs[1:]:
        assert a == a1
        dx = x - x1
        dx[:, 2] = np.mod(dx[:, 2] + 0.5, 1.0) - 0.5
        disp = np.abs(x1 - d["pos"])
        disp[:, 2] = np.minimum(disp[:, 2], 1.0 - disp[:, 2])
        assert np.abs(dx).max() <= 1e-5 * disp.max()
        assert np.abs(v - v1).max() <= 1e-5 * np.abs(dv1).max()
    # the same world size twice: the same bits
    np.testing.assert_array_equal(runs[2][0], runs[3][0])
    np.testing.assert_array_equal(runs[2][1], runs[3][1])


def test_sharded_context_refuses_whole_state_calls(env):
    torch, sc, shard = env
    w, d, t0, dt = load(n=300)
    stream = torch.cuda.current_stream().cuda_stream
    sim = sc.Simulation(config(sc, w, t0, sc.STEPS_FP32_KAHAN, stream), d["pos"], d["vel"], d["m"], d["h"])
    with pytest.raises(sc.StepsError):
        sc.steps_cyl_shard(sim.ctx, 0, 4)            # 300 rows are 3 blocks: at most 3 ranks
    rows = shard.GpuRows(sim, 1, 2, symmetric=False)
    for call in (lambda: sim.step(dt, 1), lambda: sim.forces_subset(np.arange(4)),
                 lambda: sc.steps_cyl_shard(sim.ctx, 0, 2),
                 lambda: sc.steps_cyl_shard_kick(sim.ctx, rows.send)):   # no drift before the kick
        with pytest.raises(sc.StepsError) as e:
            call()
        assert e.value.code == sc.STEPS_EINVAL
    rows.drift(dt)
    with pytest.raises(sc.StepsError):
        sim.forces()                                 # half a step is done
    sim.close()


def test_sharded_simulation_over_a_one_rank_nccl_group(env):
    # ShardedSimulation's own exchange (NCCL all-gather into one tensor) on a
    # one-rank process group: equal to the unsharded KDK bit for bit
    torch, sc, shard = env
    import torch.distributed as dist
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        w, d, t0, dt = load(n=700, seed=53)
        stream = torch.cuda.current_stream().cuda_stream
        cfg = config(sc, w, t0, sc.STEPS_FP32_KAHAN, stream)
        ref = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
        ref.step(dt, 3)
        x_ref, v_ref, _, _ = ref.state()
        dg_ref = ref.diagnostics()
        ref.close()
        sim = shard.ShardedSimulation(shard.GpuRows(sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"]), 0, 1))
        sim.step(dt, 3)
        st = sim.state()
        np.testing.assert_array_equal(st[:, :3], x_ref)
        np.testing.assert_array_equal(st[:, 3:], v_ref)
        dg = sim.diagnostics()
        np.testing.assert_array_equal(dg[:6], dg_ref[[0, 1, 2, 3, 4, 7]])
        sim.compute.sim.close()
    finally:
        dist.destroy_process_group()
