"""GPU tests of the correction-table tail (STEPS_TAIL_TABLE) against the FP64
oracle: the GPU-built table against the oracle's nodes, the table form against
the oracle's table form and against the exact windowed image sum, errors and
fallback, and a KDK run with periodic checks and checkpoint/resume."""
import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics
from tests.gpu_helpers import oracle_accel, stats, table_dR_max

pytestmark = pytest.mark.gpu

N_CUT, N0 = 64, 4


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


@pytest.fixture(scope="module")
def tabled(sc):
    w, d = workload()
    cfg = sc.Config(n_cut=N_CUT, n0=N0, precision=sc.STEPS_FP32_KAHAN, rho_bar=w.rho_bar, check_particles=512)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    rep = sc.steps_cyl_build_tail_table(sim.ctx, 257, 33)
    yield w, d, sim, rep
    sim.close()


def test_table_nodes_match_oracle(sc, tabled):
    _, d, sim, rep = tabled
    print("build report", rep)
    assert rep[2] == 1.0 and rep[0] <= 1e-6   # both forms carry FP32 rounding of ~1e-7
    tab, lib_dR_max = sc.steps_cyl_get_tail_table(sim.ctx)
    dR_max = table_dR_max(d["pos"])
    assert lib_dR_max == pytest.approx(dR_max, rel=1e-15)
    ref = oracle.tail_table_build(oracle.make_table_cfg(N_CUT, N0, tab.shape[1], tab.shape[0], dR_max))
    assert np.abs(tab - ref).max() <= 1e-6 * np.abs(ref).max()
    assert np.allclose(tab, ref, rtol=2e-7, atol=1e-9 * np.abs(ref).max())


def test_table_form_matches_oracle_table_form(sc, tabled):
    w, d, sim, _ = tabled
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    a = sim.forces()
    tab, lib_dR_max = sc.steps_cyl_get_tail_table(sim.ctx)
    dR_max = table_dR_max(d["pos"])
    assert lib_dR_max == pytest.approx(dR_max, rel=1e-15)
    cfg = oracle.make_table_cfg(N_CUT, N0, tab.shape[1], tab.shape[0], dR_max)
    idx = ics.subsample(d["m"].shape[0], 128, seed=11)
    ref = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, oracle.tail_table_build(cfg), cfg, idx=idx)
    ref += oracle.background_field(d["pos"][idx], ics.R_SIM, N_CUT * 1.0, 1.0, w.rho_bar, mode=1)
    med, p999, mx = stats(a[idx], ref)
    print(f"table kernel vs oracle table form: median {med:.2e} max {mx:.2e}")
    assert med <= 1e-6 and mx <= 1e-4
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_FULL)


def test_table_form_against_exact_sum(sc, tabled):
    w, d, sim, _ = tabled
    idx = ics.subsample(d["m"].shape[0], 160, seed=12)
    exact = oracle_accel(d["pos"], d["m"], d["h"], N_CUT, idx=idx, rho0=w.rho_bar)
    plain = stats(sim.forces()[idx], exact)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    tabf = stats(sim.forces()[idx], exact)
    print(f"vs exact: plain median {plain[0]:.2e} p99.9 {plain[1]:.2e}; table median {tabf[0]:.2e} p99.9 {tabf[1]:.2e}")
    assert tabf[0] <= 1e-5 and tabf[1] <= 1e-3
    assert tabf[0] <= 3 * plain[0] + 1e-8   # the table adds nothing visible to the FP32 error
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_FULL)


def test_table_errors_and_rejection(sc):
    w, d = workload(600, 4)
    sim = sc.Simulation(sc.Config(n_cut=N_CUT, n0=N0, rho_bar=w.rho_bar), d["pos"], d["vel"], d["m"], d["h"])
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    assert e.value.code == sc.STEPS_ENOSURROGATE
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_build_tail_table(sim.ctx, 1, 33)
    assert e.value.code == sc.STEPS_EINVAL
    # bounds no form can meet: rejected, the table is not used
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_build_tail_table(sim.ctx, 33, 5, err_median=1e-30, err_p999=1e-30, check_particles=64)
    assert e.value.code == sc.STEPS_ESURROGATE_REJECTED
    with pytest.raises(sc.StepsError):
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    sc.steps_cyl_build_tail_table(sim.ctx, 65, 9, check_particles=64)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    sim.set_precision(sc.STEPS_FP64)          # FP64 selects the full sum
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    assert e.value.code == sc.STEPS_EINVAL
    sim.close()


def test_kdk_with_table_checks_and_resume(sc, tmp_path):
    w, d = workload(2000, 6)
    t0, dt = ics.run_schedule(ics.WORKLOADS["production_n524288"])
    cfg = sc.Config(n_cut=N_CUT, n0=N0, rho_bar=w.rho_bar, comoving=True, a_start=0.02, t_start=t0, check_every=3,
                    check_particles=256)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    sc.steps_cyl_build_tail_table(sim.ctx, 257, 33, check_particles=256)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    d0 = sim.diagnostics()
    sim.step(dt, 7)                            # two periodic checks pass
    rep = sc.steps_cyl_check_tail(sim.ctx, sc.STEPS_TAIL_TABLE, 256)
    assert rep[0] <= 1e-5 and rep[1] <= 1e-3
    path = str(tmp_path / "table.ckpt")
    sim.checkpoint(path)
    sim.step(dt, 4)
    xa, va, aa, ta = sim.state()
    res = sc.Simulation.resume(path)
    res.step(dt, 4)
    xb, vb, ab, tb = res.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and aa == ab and ta == tb
    d1 = sim.diagnostics()
    pscale = np.sum(d["m"][:, None] * np.abs(va)) * aa ** 2   # canonical momentum scale
    assert pscale > 0 and abs(d1[2] - d0[2]) < 1e-6 * pscale
    res.close()
    sim.close()
