"""GPU parity of the KDK integrator (Sect. 2.1) and its conservation laws,
against the oracle's KDK, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20787_gb300 import steps_cyl
    steps_cyl.load()
    return steps_cyl


def wrapped_diff(a, b, L=1.0):
    d = a - b
    d[:, 2] = np.mod(d[:, 2] + 0.5 * L, L) - 0.5 * L
    return d


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-6)])
def test_static_kdk_matches_oracle(sc, precision, tol):
    n, n_cut, dt, steps = 512, 16, 1e-3, 10
    d = ics.particle_load(n, 0, 1.0)
    rho0 = d["m"].sum() / (np.pi * ics.R_SIM ** 2)
    c = oracle.make_cosmo(comoving=False)
    xo, po, _, _ = oracle.kdk(d["pos"], d["vel"], d["m"], d["h"], 1.0, 1.0, n_cut, ics.R_SIM, rho0, 1, c, 1.0, 0.0,
                              dt, steps)
    sim = sc.Simulation(sc.Config(n_cut=n_cut, precision=precision), d["pos"], d["vel"], d["m"], d["h"])
    sim.step(dt, steps)
    xg, vg, a, t = sim.state()
    assert a == 1.0 and t == pytest.approx(steps * dt)
    disp = np.abs(wrapped_diff(xo, d["pos"])).max()
    assert np.abs(wrapped_diff(xg, xo)).max() <= tol * max(disp, 1e-12) * 10 + 1e-15
    assert np.abs(vg - po).max() <= tol * np.abs(po).max() * 10
    sim.close()


def test_comoving_kdk_matches_oracle(sc):
    w = ics.WORKLOADS["lcdm_n65536"]
    n, steps = 384, 6
    d = ics.particle_load(n, 1, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    t0, dt = ics.run_schedule(w)
    c = oracle.make_cosmo()
    xo, po, ao, to = oracle.kdk(d["pos"], d["vel"], d["m"], d["h"], 1.0, 1.0, w.n_cut, ics.R_SIM, w.rho_bar, 1, c,
                                w.a_start, t0, dt, steps)
    cfg = sc.Config(n_cut=w.n_cut, precision=0, comoving=True, a_start=w.a_start, t_start=t0, rho_bar=w.rho_bar)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    sim.step(dt, steps)
    xg, vg, a, t = sim.state()
    assert a == pytest.approx(ao, rel=1e-14)
    assert t == pytest.approx(to, rel=1e-14)
    disp = np.abs(wrapped_diff(xo, d["pos"])).max()
    assert np.abs(wrapped_diff(xg, xo)).max() <= 1e-10 * disp
    vo = po / ao ** 2  # oracle holds canonical momenta
    assert np.abs(vg - vo).max() <= 1e-10 * np.abs(vo).max()
    sim.close()


def test_conservation_over_many_steps(sc):
    w = ics.WORKLOADS["lcdm_n65536"]
    d = ics.particle_load(4096, 11, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    d["vel"] = np.random.default_rng(0).normal(0.0, 0.01, (4096, 3))
    t0, dt = ics.run_schedule(w)
    cfg = sc.Config(n_cut=w.n_cut, precision=1, comoving=True, a_start=w.a_start, t_start=t0, rho_bar=w.rho_bar)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    d0 = sim.diagnostics()
    sim.step(dt, 20)
    d1 = sim.diagnostics()
    scale = np.sum(d["m"][:, None] * np.abs(d["vel"])) * w.a_start ** 2
    assert abs(d1[2] - d0[2]) < 1e-6 * scale       # P_z (canonical)
    assert abs(d1[3] - d0[3]) < 1e-6 * scale * 4   # L_z
    assert d1[5] > d0[5] and d1[7] == pytest.approx(w.M_tot, rel=1e-12)
    sim.close()


def test_set_state_and_restart_bit_identical(sc):
    d = ics.particle_load(1000, 3, 1.0)
    cfg = sc.Config(n_cut=8, precision=1)
    s1 = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    s1.step(1e-3, 6)
    x_mid, v_mid, _, _ = s1.state()
    s1.step(1e-3, 4)
    x_end, v_end, _, _ = s1.state()
    s2 = sc.Simulation(cfg, x_mid, v_mid, d["m"], d["h"])
    s2.step(1e-3, 4)
    x2, v2, _, _ = s2.state()
    np.testing.assert_array_equal(x2, x_end)
    np.testing.assert_array_equal(v2, v_end)
    s1.close()
    s2.close()
