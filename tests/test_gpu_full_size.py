"""Parity at the full sizes of the benchmark workloads, in the launch
configuration the benchmark times (the stream-K pair kernels over all N
particles), on seeded samples of i that the FP64 oracle computes one by one.
Gates: relative force error <= 1e-5 at the median and <= 1e-3 at the 99.9th
percentile for every FP32 form and for the learned tail."""
import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics
from tests.gpu_helpers import oracle_accel, seeded_surrogate, stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20787_gb300 import steps_cyl
    steps_cyl.load()
    return steps_cyl


def full_sim(sc, w, d, **kw):
    cfg = sc.Config(n_cut=w.n_cut, rho_bar=w.rho_bar, **kw)
    return sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])


@pytest.mark.parametrize("name, forms", [("precision_n262144", ("kahan", "plain")),
                                         ("production_n524288", ("kahan",))])
def test_full_size_fp32_forms(sc, name, forms):
    w = ics.WORKLOADS[name]
    d = ics.workload_ics(w)
    idx = ics.subsample(w.n, 192, seed=2024)
    ref = oracle_accel(d["pos"], d["m"], d["h"], w.n_cut, idx=idx, rho0=w.rho_bar)
    sim = full_sim(sc, w, d, precision=sc.STEPS_FP32_KAHAN)
    for form in forms:
        sim.set_precision(sc.STEPS_FP32_KAHAN if form == "kahan" else sc.STEPS_FP32_PLAIN)
        med, p999, mx = stats(sim.forces()[idx], ref)
        print(f"{name} FP32-{form}: median {med:.2e} p99.9 {p999:.2e} max {mx:.2e}")
        assert med <= 1e-5 and p999 <= 1e-3
    sim.close()


def test_full_size_surrogate(sc):
    # N = 2^20, Ncut = 64, n0 = 4: the plain 128-image sum and the learned tail
    # (trained on the GPU) against the FP64 oracle, and the surrogate kernel with
    # a seeded network against the oracle's own statement of the surrogate form
    w = ics.WORKLOADS["surrogate_n1048576"]
    d = ics.workload_ics(w)
    sim = full_sim(sc, w, d, n0=w.n0, precision=sc.STEPS_FP32_KAHAN)
    report = sc.steps_cyl_train_surrogate(sim.ctx, sc.steps_cyl_train_cfg_default())
    assert report[4] == 1.0
    idx = ics.subsample(w.n, 96, seed=77)
    exact = oracle_accel(d["pos"], d["m"], d["h"], w.n_cut, idx=idx, rho0=w.rho_bar)
    med, p999, _ = stats(sim.forces()[idx], exact)
    print(f"N=2^20 plain FP32-Kahan: median {med:.2e} p99.9 {p999:.2e}")
    assert med <= 1e-5 and p999 <= 1e-3
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    a = sim.forces()
    med, p999, _ = stats(a[idx], exact)
    print(f"N=2^20 learned tail vs exact: median {med:.2e} p99.9 {p999:.2e}")
    assert med <= 1e-5 and p999 <= 1e-3
    sub = idx[:32]
    w16, cfg = seeded_surrogate(sc, sim.ctx, 43, w.n_cut, w.n0)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    a = sim.forces()
    ref = oracle.pair_field_surrogate(d["pos"], d["m"], d["h"], 1.0, 1.0, w16, cfg, idx=sub)
    ref += oracle.background_field(d["pos"][sub], ics.R_SIM, w.n_cut * 1.0, 1.0, w.rho_bar, mode=1)
    med, _, mx = stats(a[sub], ref)
    print(f"N=2^20 surrogate kernel (seeded network) vs oracle surrogate form: median {med:.2e} max {mx:.2e}")
    assert med <= 2e-6 and mx <= 1e-4
    # the correction-table tail on the same particles
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_FULL)
    sc.steps_cyl_build_tail_table(sim.ctx, 257, 33)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    med, p999, _ = stats(sim.forces()[idx], exact)
    print(f"N=2^20 table tail vs exact: median {med:.2e} p99.9 {p999:.2e}")
    assert med <= 1e-5 and p999 <= 1e-3
    sim.close()
