"""GPU tests of the triangular-shaped-cloud (TSC) read of the correction table
(Sect. 2.3: CIC or TSC), against the FP64 oracle's TSC read: the table form of
a finite and of the infinite window against the oracle's TSC table form and
against the exact image sums, the acceptance check run in the chosen read,
the read kept by a table built earlier, a bit-identical checkpoint/resume, and
the refused values."""
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
def tsc_sim(sc):
    w, d = workload()
    cfg = sc.Config(n_cut=N_CUT, n0=N0, precision=sc.STEPS_FP32_KAHAN, rho_bar=w.rho_bar, check_particles=512)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    sc.steps_cyl_set_table_read(sim.ctx, sc.STEPS_TABLE_READ_TSC)
    rep = sc.steps_cyl_build_tail_table(sim.ctx, 257, 33)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    yield w, d, sim, rep
    sim.close()


def test_check_runs_in_the_tsc_read(sc, tsc_sim):
    *_, rep = tsc_sim
    print("TSC build report", rep)
    assert rep[2] == 1.0 and rep[0] <= 1e-5 and rep[1] <= 1e-3


def test_tsc_form_matches_oracle_tsc_form(sc, tsc_sim):
    w, d, sim, _ = tsc_sim
    a = sim.forces()
    tab, dR_max = sc.steps_cyl_get_tail_table(sim.ctx)
    assert dR_max == pytest.approx(table_dR_max(d["pos"]), rel=1e-15)
    cfg = oracle.make_table_cfg(N_CUT, N0, tab.shape[1], tab.shape[0], dR_max, read=oracle.TABLE_TSC)
    idx = ics.subsample(d["m"].shape[0], 128, seed=11)
    ref = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, oracle.tail_table_build(cfg), cfg, idx=idx)
    ref += oracle.background_field(d["pos"][idx], ics.R_SIM, N_CUT, 1.0, w.rho_bar)
    med, _, mx = stats(a[idx], ref)
    print(f"TSC table kernel vs oracle TSC table form: median {med:.2e} max {mx:.2e}")
    assert med <= 1e-6 and mx <= 1e-4
    # and the TSC read differs from the CIC read by more than that (it smooths)
    cic = oracle.make_table_cfg(N_CUT, N0, tab.shape[1], tab.shape[0], dR_max)
    ref_cic = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, oracle.tail_table_build(cic), cic, idx=idx)
    ref_cic += oracle.background_field(d["pos"][idx], ics.R_SIM, N_CUT, 1.0, w.rho_bar)
    assert np.abs(ref_cic - ref).max() > 0


def test_tsc_form_against_exact_sum(sc, tsc_sim):
    w, d, sim, _ = tsc_sim
    idx = ics.subsample(d["m"].shape[0], 160, seed=12)
    exact = oracle_accel(d["pos"], d["m"], d["h"], N_CUT, idx=idx, rho0=w.rho_bar)
    med, p999, _ = stats(sim.forces()[idx], exact)
    print(f"TSC table form vs exact windowed sum: median {med:.2e} p99.9 {p999:.2e}")
    assert med <= 1e-5 and p999 <= 1e-3


def test_built_table_keeps_its_read(sc, tsc_sim):
    _, _, sim, _ = tsc_sim
    a0 = sim.forces()
    sc.steps_cyl_set_table_read(sim.ctx, sc.STEPS_TABLE_READ_CIC)   # applies to the next build only
    assert np.array_equal(sim.forces(), a0)
    sc.steps_cyl_set_table_read(sim.ctx, sc.STEPS_TABLE_READ_TSC)
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_set_table_read(sim.ctx, 2)
    assert e.value.code == sc.STEPS_EINVAL


def test_infinite_window_tsc_against_oracle(sc):
    w, d = workload(2500, 8)
    cfg = sc.Config(n_cut=0, n0=N0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_TABLE,
                    background=sc.STEPS_BG_INFINITE, rho_bar=w.rho_bar)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    sc.steps_cyl_set_table_read(sim.ctx, sc.STEPS_TABLE_READ_TSC)
    sc.steps_cyl_build_tail_table_ewald(sim.ctx, 144, 128)
    a = sim.forces()
    tab, dR_max = sc.steps_cyl_get_tail_table(sim.ctx)
    ocfg = oracle.make_table_cfg(0, N0, 144, 128, dR_max, read=oracle.TABLE_TSC)
    idx = ics.subsample(d["m"].shape[0], 128, seed=14)
    bg = oracle.background_field(d["pos"][idx], ics.R_SIM, 0.0, 1.0, w.rho_bar, mode=2)
    ref = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, oracle.tail_table_build(ocfg), ocfg,
                                  idx=idx) + bg
    med, _, mx = stats(a[idx], ref)
    assert med <= 1e-6 and mx <= 1e-4, (med, mx)
    exact = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx) + bg
    med, p999, _ = stats(a[idx], exact)
    print(f"infinite window, TSC read of the Ewald table vs exact line: median {med:.2e} p99.9 {p999:.2e}")
    assert med <= 1e-5 and p999 <= 1e-3
    sim.close()


def test_checkpoint_keeps_the_tsc_read(sc, tmp_path):
    w, d = workload(1500, 9)
    t0, dt = ics.run_schedule(ics.WORKLOADS["production_n524288"])
    cfg = sc.Config(n_cut=N_CUT, n0=N0, rho_bar=w.rho_bar, comoving=True, a_start=0.02, t_start=t0,
                    check_particles=256)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    sc.steps_cyl_set_table_read(sim.ctx, sc.STEPS_TABLE_READ_TSC)
    sc.steps_cyl_build_tail_table(sim.ctx, 129, 17, check_particles=256)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    sim.step(dt, 2)
    path = str(tmp_path / "tsc.ckpt")
    sim.checkpoint(path)
    sim.step(dt, 3)
    xa, va, aa, ta = sim.state()
    res = sc.Simulation.resume(path)
    res.step(dt, 3)
    xb, vb, ab, tb = res.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and aa == ab and ta == tb
    res.close()
    sim.close()
