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
    # a new context built from a saved state continues bit-identically when it
    # keeps the caller's particle order (the sum order then matches)
    d = ics.particle_load(1000, 3, 1.0)
    cfg = sc.Config(n_cut=8, precision=1, reorder_every=-1)
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


def test_internal_order_is_invisible(sc):
    d = ics.particle_load(3000, 13, 1.0)
    d["vel"] = np.random.default_rng(5).normal(0.0, 0.02, (3000, 3))
    plain = sc.Simulation(sc.Config(n_cut=8, precision=1, reorder_every=-1), d["pos"], d["vel"], d["m"], d["h"])
    sorted_ = sc.Simulation(sc.Config(n_cut=8, precision=1, reorder_every=3), d["pos"], d["vel"], d["m"], d["h"])
    x0, v0, _, _ = sorted_.state()
    np.testing.assert_array_equal(x0, d["pos"])
    np.testing.assert_allclose(v0, d["vel"], rtol=0, atol=0)
    a1, a2 = plain.forces(), sorted_.forces()
    # the two orders sum the same pair forces in different orders: they agree
    # to FP32 rounding (the FP32 forms' own error against the oracle is larger)
    r = np.linalg.norm(a1 - a2, axis=1) / np.linalg.norm(a1, axis=1)
    assert np.median(r) < 1e-6 and r.max() < 1e-4
    plain.step(1e-3, 7)
    sorted_.step(1e-3, 7)   # re-ordered twice on the way
    xa, va, _, _ = plain.state()
    xb, vb, _, _ = sorted_.state()
    assert np.abs(wrapped_diff(xa, xb)).max() < 1e-9
    assert np.abs(va - vb).max() < 1e-6 * np.abs(va).max()
    plain.close()
    sorted_.close()


def test_set_state_moves_masses_with_the_new_order(sc):
    d1 = ics.particle_load(900, 21, 1.0)
    d2 = ics.particle_load(900, 22, 1.0)   # different positions, same masses/softenings below
    sim = sc.Simulation(sc.Config(n_cut=6, precision=0), d1["pos"], d1["vel"], d1["m"], d1["h"])
    cols = [np.ascontiguousarray(d2["pos"][:, k]) for k in range(3)] + [np.zeros(900)] * 3
    sc.steps_cyl_set_state(sim.ctx, *cols)
    ref = oracle.pair_field(d2["pos"], d1["m"], d1["h"], 1.0, 1.0, 6)
    rho0 = d1["m"].sum() / (np.pi * ics.R_SIM ** 2)
    ref += oracle.background_field(d2["pos"], ics.R_SIM, 6.0, 1.0, rho0, mode=1)
    a = sim.forces()
    r = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert r.max() < 1e-10
    sim.close()


def test_checkpoint_resume_is_bit_identical(sc, tmp_path):
    # re-ordering every 3 steps and a comoving background: the checkpoint must
    # carry the internal order, the counters, the table and the cached forces
    w = ics.WORKLOADS["lcdm_n65536"]
    d = ics.particle_load(1500, 17, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    t0, dt = ics.run_schedule(w)
    cfg = sc.Config(n_cut=8, precision=1, comoving=True, a_start=0.02, t_start=t0, rho_bar=w.rho_bar, reorder_every=3)
    s1 = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    s1.step(dt, 5)
    path = str(tmp_path / "state.ckpt")
    s1.checkpoint(path)
    s1.step(dt, 4)
    x1, v1, a1, t1 = s1.state()
    s2 = sc.Simulation.resume(path)
    s2.step(dt, 4)
    x2, v2, a2, t2 = s2.state()
    np.testing.assert_array_equal(x2, x1)
    np.testing.assert_array_equal(v2, v1)
    assert (a2, t2) == (a1, t1)
    with open(path, "r+b") as fh:
        fh.write(b"NOTSTEPS")
    with pytest.raises(sc.StepsError):
        sc.Simulation.resume(path)
    s1.close()
    s2.close()


def test_diagnostics_match_oracle(sc):
    # Sect. 1 diagnostics of a state on the oracle's own comoving trajectory:
    # a context is given the oracle's state after a few KDK steps, and its
    # diagnostics must equal the oracle's sums of that state; then a context
    # stepped by the library from the start must reach the oracle's values to
    # the KDK parity tolerance.
    w = ics.WORKLOADS["lcdm_n65536"]
    n, steps = 384, 6
    d = ics.particle_load(n, 7, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    vel = np.random.default_rng(17).normal(0.0, 0.05, (n, 3))
    t0, dt = ics.run_schedule(w)
    c = oracle.make_cosmo()
    xo, po, ao, to = oracle.kdk(d["pos"], vel * w.a_start ** 2, d["m"], d["h"], 1.0, 1.0, w.n_cut, ics.R_SIM,
                                w.rho_bar, 1, c, w.a_start, t0, dt, steps)
    do = oracle.diagnostics(xo, po, d["m"], ao)
    pscale = np.sum(d["m"][:, None] * np.abs(po))
    lscale = np.sum(d["m"] * np.hypot(xo[:, 0], xo[:, 1]) * np.linalg.norm(po, axis=1))

    cfg = sc.Config(n_cut=w.n_cut, precision=0, comoving=True, a_start=ao, t_start=to, rho_bar=w.rho_bar)
    held = sc.Simulation(cfg, xo, po / ao ** 2, d["m"], d["h"])
    dg = held.diagnostics()
    held.close()
    assert dg[5] == ao and dg[6] == to
    np.testing.assert_allclose(dg[0:3], do[0:3], rtol=0, atol=1e-12 * pscale)
    assert abs(dg[3] - do[3]) <= 1e-12 * lscale
    assert dg[4] == pytest.approx(do[4], rel=1e-12)
    assert dg[7] == pytest.approx(do[5], rel=1e-14)

    cfg = sc.Config(n_cut=w.n_cut, precision=0, comoving=True, a_start=w.a_start, t_start=t0, rho_bar=w.rho_bar)
    sim = sc.Simulation(cfg, d["pos"], vel, d["m"], d["h"])
    sim.step(dt, steps)
    ds = sim.diagnostics()
    sim.close()
    np.testing.assert_allclose(ds[0:3], do[0:3], rtol=0, atol=1e-10 * pscale)
    assert abs(ds[3] - do[3]) <= 1e-10 * lscale
    assert ds[4] == pytest.approx(do[4], rel=1e-9)
    assert ds[5] == pytest.approx(ao, rel=1e-14)
