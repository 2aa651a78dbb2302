"""GPU tests of the learned far-image surrogate (training kernels, fused FP16
mma inference, acceptance and fallback) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics
from tests.gpu_helpers import oracle_accel, seeded_surrogate, stats

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


def test_tail_sums_match_oracle(sc):
    rng = np.random.default_rng(0)
    smp = np.stack([rng.uniform(0, 8, 300), rng.uniform(-0.5, 0.5, 300), rng.uniform(0.01, 10.0, 300)], 1)
    smp[:5, 0] = [0.0, 1e-3, 0.5, 4.4, 7.9]
    got = sc.steps_cyl_tail_sums(smp, N_CUT, N0)
    for s in range(smp.shape[0]):
        ref = oracle.tail_sums(smp[s, 0], smp[s, 1], smp[s, 2], 1.0, N_CUT, N0)
        assert got[s, 0] == pytest.approx(ref[0], rel=1e-12, abs=1e-16)
        assert got[s, 1] == pytest.approx(ref[1], rel=1e-11, abs=1e-15)


def test_mlp_gradients_match_oracle(sc):
    rng = np.random.default_rng(1)
    w = rng.normal(0, 0.3, sc.STEPS_SURR_NW).astype(np.float32)
    u = rng.uniform(-1, 1, (257, 3)).astype(np.float32)
    t = rng.normal(0, 1, (257, 2)).astype(np.float32)
    loss, g = sc.steps_cyl_mlp_loss_grad(w, u, t)
    lref, gref = oracle.mlp_loss_grad(w.astype(np.float64), u.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(lref, rel=1e-5)
    assert np.abs(g - gref).max() <= 2e-5 * np.abs(gref).max()


def small_workload(n=4096, seed=3):
    w = ics.WORKLOADS["surrogate_n1048576"]
    d = ics.particle_load(n, seed, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    return w, d


@pytest.fixture(scope="module")
def trained(sc):
    w, d = small_workload()
    cfg = sc.Config(n_cut=N_CUT, n0=N0, precision=sc.STEPS_FP32_KAHAN, rho_bar=w.rho_bar, comoving=True,
                    a_start=0.02, check_particles=512)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    tcfg = sc.steps_cyl_train_cfg_default(n_samples=1 << 18, epochs=40, check_particles=512)
    report = sc.steps_cyl_train_surrogate(sim.ctx, tcfg)
    params = sc.steps_cyl_get_surrogate(sim.ctx)
    yield w, d, sim, report, params
    sim.close()


def test_training_is_accepted(trained):
    _, _, _, report, params = trained
    print("train report", report)
    assert report[4] == 1.0
    assert report[1] < 0.05           # held-out RMS in normalised units
    assert report[2] <= 1e-5 and report[3] <= 1e-3
    assert np.all(np.isfinite(params))


def test_surrogate_kernel_matches_oracle_definition(sc, trained):
    # a seeded network, so that the oracle's inputs do not come from the library
    w, d, sim, _, params = trained
    w16, cfg = seeded_surrogate(sc, sim.ctx, 41, N_CUT, N0)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    a = sim.forces()
    sc.steps_cyl_set_surrogate(sim.ctx, params)   # the trained network again, for the other tests
    idx = ics.subsample(d["m"].shape[0], 160, seed=7)
    ref = oracle.pair_field_surrogate(d["pos"], d["m"], d["h"], 1.0, 1.0, w16, cfg, idx=idx)
    ref += oracle.background_field(d["pos"][idx], ics.R_SIM, N_CUT * 1.0, 1.0, w.rho_bar, mode=1)
    ref /= 0.02 ** 3
    med, p999, mx = stats(a[idx], ref)
    print(f"surrogate kernel vs oracle surrogate form: median {med:.2e} max {mx:.2e}")
    assert med <= 2e-6 and mx <= 1e-4


def test_surrogate_accuracy_and_gain_against_exact_sum(sc, trained):
    w, d, sim, _, params = trained
    idx = ics.subsample(d["m"].shape[0], 160, seed=8)
    exact = oracle_accel(d["pos"], d["m"], d["h"], N_CUT, idx=idx, rho0=w.rho_bar, a=0.02)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    med, p999, _ = stats(sim.forces()[idx], exact)
    # the same form with the network switched off (residual = 0): the base alone
    base = params.copy()
    base[1184:1252] = 0.0    # W3, b3, mu
    sc.steps_cyl_set_surrogate(sim.ctx, base, err_median=1.0, err_p999=1.0)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    bmed, bp999, _ = stats(sim.forces()[idx], exact)
    print(f"with network: median {med:.2e} p99.9 {p999:.2e}; base only: median {bmed:.2e} p99.9 {bp999:.2e}")
    assert med <= 1e-5 and p999 <= 1e-3
    assert med < bmed / 5
    # restore the trained network for the other tests
    sc.steps_cyl_set_surrogate(sim.ctx, params)


def test_softened_tail_images(sc):
    # softening of several L puts tail images inside the support: the kernel's
    # exact correction must agree with the oracle's definition
    w, d = small_workload(1500, 5)
    d["h"] = np.random.default_rng(2).uniform(0.5, 6.0, 1500)
    cfg = sc.Config(n_cut=N_CUT, n0=N0, precision=1, rho_bar=w.rho_bar, check_particles=256)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    w16, scfg = seeded_surrogate(sc, sim.ctx, 42, N_CUT, N0)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    a = sim.forces()
    idx = ics.subsample(1500, 100, seed=9)
    ref = oracle.pair_field_surrogate(d["pos"], d["m"], d["h"], 1.0, 1.0, w16, scfg, idx=idx)
    ref += oracle.background_field(d["pos"][idx], ics.R_SIM, N_CUT * 1.0, 1.0, w.rho_bar, mode=1)
    med, _, mx = stats(a[idx], ref)
    assert med <= 2e-6 and mx <= 1e-4
    sim.close()


def test_rejected_network_falls_back_to_plain_sum(sc, trained):
    w, d, sim, _, params = trained
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_FULL)
    plain = sim.forces()
    bad = params.copy()
    bad[:1250] += np.random.default_rng(3).normal(0, 2.0, 1250).astype(np.float32)
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_set_surrogate(sim.ctx, bad)
    assert e.value.code == sc.STEPS_ESURROGATE_REJECTED
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    assert e.value.code == sc.STEPS_ENOSURROGATE
    np.testing.assert_array_equal(sim.forces(), plain)
    nan = params.copy()
    nan[7] = np.nan
    with pytest.raises(sc.StepsError):
        sc.steps_cyl_set_surrogate(sim.ctx, nan)
    sc.steps_cyl_set_surrogate(sim.ctx, params)   # the trained network is accepted again


def test_kdk_with_surrogate_and_periodic_checks(sc, trained):
    w, d, _, _, params = trained
    t0 = ics.lcdm_time_of_a(0.02)
    dt = 2e-4
    runs = []
    for tail in (sc.STEPS_TAIL_FULL, sc.STEPS_TAIL_SURROGATE):
        cfg = sc.Config(n_cut=N_CUT, n0=N0, precision=1, rho_bar=w.rho_bar, comoving=True, a_start=0.02, t_start=t0,
                        check_every=3, check_particles=256)
        sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
        if tail == sc.STEPS_TAIL_SURROGATE:
            sc.steps_cyl_set_surrogate(sim.ctx, params)
            sc.steps_cyl_set_tail(sim.ctx, tail)
        sim.step(dt, 8)           # two periodic checks on the way
        runs.append(sim.state())
        sim.close()
    (x0, v0, a0, _), (x1, v1, a1, _) = runs
    assert a0 == a1
    dx = x1 - x0
    dx[:, 2] = np.mod(dx[:, 2] + 0.5, 1.0) - 0.5
    disp = np.abs(x0 - d["pos"])
    assert np.abs(dx).max() <= 1e-5 * max(disp.max(), 1e-12) + 1e-13
    assert np.abs(v1 - v0).max() <= 1e-4 * np.abs(v0).max()
