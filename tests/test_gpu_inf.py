"""GPU tests of the infinite window (Ncut -> infinity, Sect. 2.2: n_cut = 0),
carried by the correction table with the infinite-cylinder background of eq.
F_horiz_infty: the table built at init against the oracle's nodes, the forces
against the oracle's table form and against the exact infinite image line, the
refused combinations, a static KDK run against an FP64 KDK on the oracle's
field, and checkpoint/resume."""
import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics
from tests.gpu_helpers import seeded_surrogate, stats, table_dR_max

pytestmark = pytest.mark.gpu

N0 = 4


@pytest.fixture(scope="module")
def sc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20787_gb300 import steps_cyl
    steps_cyl.load()
    return steps_cyl


def workload(n=3000, seed=3):
    w = ics.WORKLOADS["surrogate_n1048576"]
    return w, ics.particle_load(n, seed, w.M_tot, displaced=True, rho_bar=w.rho_bar)


def inf_config(sc, rho_bar, **kw):
    base = dict(n_cut=0, n0=N0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_TABLE,
                background=sc.STEPS_BG_INFINITE, rho_bar=rho_bar)
    base.update(kw)
    return sc.Config(**base)


def background(pos, rho_bar):
    return oracle.background_field(pos, ics.R_SIM, 0.0, 1.0, rho_bar, mode=2)


@pytest.fixture(scope="module")
def infsim(sc):
    w, d = workload()
    sim = sc.Simulation(inf_config(sc, w.rho_bar), d["pos"], d["vel"], d["m"], d["h"])
    yield w, d, sim
    sim.close()


def test_inf_table_nodes_match_oracle(sc, infsim):
    _, d, sim = infsim
    tab, lib_dR_max = sc.steps_cyl_get_tail_table(sim.ctx)
    dR_max = table_dR_max(d["pos"])
    assert lib_dR_max == pytest.approx(dR_max, rel=1e-15)
    assert tab.shape == (33, 257, 2)
    ref = oracle.tail_table_build(oracle.make_table_cfg(0, N0, tab.shape[1], tab.shape[0], dR_max))
    assert np.allclose(tab, ref, rtol=2e-7, atol=1e-9 * np.abs(ref).max())


def test_inf_table_form_matches_oracle_table_form(sc, infsim):
    w, d, sim = infsim
    a = sim.forces()
    tab, lib_dR_max = sc.steps_cyl_get_tail_table(sim.ctx)
    dR_max = table_dR_max(d["pos"])
    assert lib_dR_max == pytest.approx(dR_max, rel=1e-15)
    cfg = oracle.make_table_cfg(0, N0, tab.shape[1], tab.shape[0], dR_max)
    idx = ics.subsample(d["m"].shape[0], 128, seed=11)
    ref = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, oracle.tail_table_build(cfg), cfg, idx=idx)
    ref += background(d["pos"][idx], w.rho_bar)
    med, _, mx = stats(a[idx], ref)
    print(f"infinite table kernel vs oracle table form: median {med:.2e} max {mx:.2e}")
    assert med <= 1e-6 and mx <= 1e-4


def test_inf_against_exact_infinite_sum(sc, infsim):
    w, d, sim = infsim
    idx = ics.subsample(d["m"].shape[0], 160, seed=12)
    exact = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx) + background(d["pos"][idx], w.rho_bar)
    med, p999, mx = stats(sim.forces()[idx], exact)
    print(f"infinite window vs exact line: median {med:.2e} p99.9 {p999:.2e} max {mx:.2e}")
    assert med <= 1e-5 and p999 <= 1e-3


@pytest.mark.parametrize("n", [2, 129, 1000])
def test_inf_ragged_sizes(sc, n):
    w, d = workload(n, 40 + n)
    sim = sc.Simulation(inf_config(sc, w.rho_bar, precision=sc.STEPS_FP32_PLAIN), d["pos"], d["vel"], d["m"], d["h"])
    idx = np.arange(n) if n <= 200 else ics.subsample(n, 200, seed=n)
    exact = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx) + background(d["pos"][idx], w.rho_bar)
    med, _, mx = stats(sim.forces()[idx], exact)
    assert med <= 2e-5 and mx <= 2e-3
    sim.close()


def test_inf_combinations_are_checked(sc, infsim):
    w, d = workload(200, 5)
    bad = [dict(precision=sc.STEPS_FP64), dict(tail=sc.STEPS_TAIL_FULL), dict(background=sc.STEPS_BG_FINITE),
           dict(n0=-1), dict(n0=512), dict(n0=0, tail=sc.STEPS_TAIL_SURROGATE), dict(topology=sc.STEPS_TOPO_R3),
           dict(n_cut=-1)]
    for kw in bad:
        with pytest.raises(sc.StepsError) as e:
            sc.Simulation(inf_config(sc, w.rho_bar, **kw), d["pos"], d["vel"], d["m"], d["h"])
        assert e.value.code == sc.STEPS_EINVAL, kw
    with pytest.raises(sc.StepsError) as e:     # a network is trained or loaded after init
        sc.Simulation(inf_config(sc, w.rho_bar, tail=sc.STEPS_TAIL_SURROGATE), d["pos"], d["vel"], d["m"], d["h"])
    assert e.value.code == sc.STEPS_ENOSURROGATE
    _, _, sim = infsim
    for call in (lambda: sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP64),
                 lambda: sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_FULL),
                 lambda: sc.steps_cyl_check_tail(sim.ctx, sc.STEPS_TAIL_TABLE, 64)):
        with pytest.raises(sc.StepsError) as e:
            call()
        assert e.value.code == sc.STEPS_EINVAL
    # a rebuilt table on a finer grid is kept without a check (no plain sum exists)
    rep = sc.steps_cyl_build_tail_table(sim.ctx, 513, 65)
    assert rep[2] == 1.0 and np.isnan(rep[0])
    tab, _ = sc.steps_cyl_get_tail_table(sim.ctx)
    assert tab.shape == (65, 513, 2)
    sc.steps_cyl_build_tail_table(sim.ctx, 257, 33)


def oracle_kdk_inf(pos, vel, m, h, rho_bar, dt, nsteps):
    # static space: p = v, kick dt/2, drift dt, kick dt/2 (eq. KDK with a = 1)
    x, v = pos.copy(), vel.copy()

    def field(x):
        return oracle.pair_field_inf(x, m, h, 1.0, 1.0) + background(x, rho_bar)

    g = field(x)
    for _ in range(nsteps):
        v += 0.5 * dt * g
        x += dt * v
        x[:, 2] -= np.floor(x[:, 2])
        g = field(x)
        v += 0.5 * dt * g
    return x, v


def test_inf_kdk_matches_oracle(sc, tmp_path):
    w, d = workload(300, 7)
    vel = np.random.default_rng(8).normal(0.0, 0.02, d["pos"].shape)
    dt, nsteps = 0.05, 4
    xo, vo = oracle_kdk_inf(d["pos"], vel, d["m"], d["h"], w.rho_bar, dt, nsteps)
    sim = sc.Simulation(inf_config(sc, w.rho_bar), d["pos"], vel, d["m"], d["h"])
    sim.step(dt, 2)
    path = str(tmp_path / "inf.ckpt")
    sim.checkpoint(path)
    sim.close()
    sim = sc.Simulation.resume(path)
    sim.step(dt, 2)
    xg, vg, _, t = sim.state()
    assert t == pytest.approx(dt * nsteps, rel=1e-14)
    dx = xg - xo
    dx[:, 2] -= np.round(dx[:, 2])
    moved = np.abs(xo - d["pos"])
    moved[:, 2] = np.minimum(moved[:, 2], 1.0 - moved[:, 2])
    print(f"KDK: max position difference {np.abs(dx).max():.2e} of max displacement {moved.max():.2e}")
    assert np.abs(dx).max() <= 2e-4 * moved.max()
    assert np.abs(vg - vo).max() <= 2e-4 * np.abs(vo - vel).max()
    tab, _ = sc.steps_cyl_get_tail_table(sim.ctx)
    assert tab.shape == (33, 257, 2)   # the resumed context rebuilt its table
    sim.close()


def test_inf_full_size_sampled(sc):
    # the benchmarked configuration (N = 65,536, FP32-Kahan), sampled particles
    w = ics.WORKLOADS["surrogate_n65536"]
    d = ics.workload_ics(w)
    sim = sc.Simulation(inf_config(sc, w.rho_bar), d["pos"], d["vel"], d["m"], d["h"])
    idx = ics.subsample(w.n, 48, seed=21)
    exact = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx) + background(d["pos"][idx], w.rho_bar)
    med, _, mx = stats(sim.forces()[idx], exact)
    print(f"N = {w.n} infinite window vs exact line: median {med:.2e} max {mx:.2e}")
    assert med <= 1e-5 and mx <= 1e-3
    sim.close()


# ---- the learned tail trained to infinity --------------------------------

def test_inf_tail_sums_match_oracle(sc):
    smp = ics.tail_training_inputs(2000, 6, 6.0, 7.0)
    smp[::2, 1] *= -1.0
    out = sc.steps_cyl_tail_sums(smp, 0, N0)
    for s in range(0, 2000, 37):
        ref = oracle.image_sums_inf(smp[s, 0], smp[s, 1], smp[s, 2], N0)
        assert out[s, 0] == pytest.approx(ref[0], rel=1e-12)
        assert out[s, 1] == pytest.approx(ref[1], rel=1e-11, abs=1e-15)


def test_inf_surrogate_kernel_matches_oracle_definition(sc, infsim):
    w, d, sim = infsim
    w16, cfg = seeded_surrogate(sc, sim.ctx, 31, 0, N0)   # checked against the table form on the way in
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    a = sim.forces()
    idx = ics.subsample(d["m"].shape[0], 128, seed=13)
    ref = oracle.pair_field_surrogate(d["pos"], d["m"], d["h"], 1.0, 1.0, w16, cfg, idx=idx)
    ref += background(d["pos"][idx], w.rho_bar)
    med, _, mx = stats(a[idx], ref)
    print(f"infinite surrogate kernel vs oracle definition: median {med:.2e} max {mx:.2e}")
    assert med <= 2e-6 and mx <= 1e-4
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)


def test_inf_softened_tail_images(sc):
    # softenings of several L put tail images inside the support of the infinite window
    w, d = workload(1500, 5)
    d["h"] = np.random.default_rng(2).uniform(0.5, 6.0, 1500)
    sim = sc.Simulation(inf_config(sc, w.rho_bar, precision=sc.STEPS_FP32_PLAIN), d["pos"], d["vel"], d["m"], d["h"])
    w16, cfg = seeded_surrogate(sc, sim.ctx, 32, 0, N0)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    idx = ics.subsample(1500, 100, seed=9)
    ref = oracle.pair_field_surrogate(d["pos"], d["m"], d["h"], 1.0, 1.0, w16, cfg, idx=idx)
    ref += background(d["pos"][idx], w.rho_bar)
    med, _, mx = stats(sim.forces()[idx], ref)
    assert med <= 2e-6 and mx <= 1e-4
    sim.close()


def test_inf_surrogate_training_and_accuracy(sc):
    w, d = workload(3000, 3)
    sim = sc.Simulation(inf_config(sc, w.rho_bar, check_particles=512, check_every=3), d["pos"], d["vel"], d["m"],
                        d["h"])
    tcfg = sc.steps_cyl_train_cfg_default(n_samples=1 << 18, epochs=40, check_particles=512)
    rep = sc.steps_cyl_train_surrogate(sim.ctx, tcfg)
    print("infinite-window training report", rep)
    assert rep[4] == 1.0 and rep[2] <= 1e-5 and rep[3] <= 1e-3
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    idx = ics.subsample(3000, 160, seed=12)
    exact = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx) + background(d["pos"][idx], w.rho_bar)
    med, p999, mx = stats(sim.forces()[idx], exact)
    print(f"trained infinite surrogate vs exact line: median {med:.2e} p99.9 {p999:.2e} max {mx:.2e}")
    assert med <= 1e-5 and p999 <= 1e-3
    chk = sc.steps_cyl_check_surrogate(sim.ctx, 256)
    assert chk[0] <= 1e-5 and chk[1] <= 1e-3
    # KDK with periodic checks against the table form
    cfg_dt = 0.02
    sim.step(cfg_dt, 6)
    assert sim.state()[3] == pytest.approx(6 * cfg_dt, rel=1e-14)
    sim.close()


def test_inf_rejected_network_keeps_the_table(sc, infsim):
    w, d, sim = infsim
    p = ics.random_surrogate_params(33, 8.0, sc=(50.0, 50.0))   # a network scaled far off the tail
    before = sim.forces()
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_set_surrogate(sim.ctx, p)
    assert e.value.code == sc.STEPS_ESURROGATE_REJECTED
    with pytest.raises(sc.StepsError):
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    np.testing.assert_array_equal(sim.forces(), before)
