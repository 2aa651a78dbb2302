"""GPU tests of the R^3 topology (eq. NewtonianForce with the radial term of
Sect. 2.1) and of glass making (Sect. 3.1: a comoving run with repulsive
gravity, G < 0, whose Hubble drag settles the load), against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics
from tests.gpu_helpers import stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20787_gb300 import steps_cyl
    steps_cyl.load()
    return steps_cyl


def ball(n, seed, R=2.0):
    d = ics.ball_load(n, seed, R)
    return d["pos"], d["m"], d["h"], d["rho_bar"]


def r3_sim(sc, pos, m, h, rho, precision, background, **kw):
    cfg = sc.Config(topology=sc.STEPS_TOPO_R3, n_cut=1, precision=precision, background=background, rho_bar=rho,
                    R_sim=2.0, **kw)
    return sc.Simulation(cfg, pos, np.zeros_like(pos), m, h)


@pytest.mark.parametrize("precision, med_gate, max_gate", [(0, 1e-12, 1e-10), (1, 2e-6, 1e-4), (2, 1e-5, 1e-3)])
@pytest.mark.parametrize("background", [0, 3])
def test_r3_forces_match_oracle(sc, precision, med_gate, max_gate, background):
    pos, m, h, rho = ball(2000, 1)
    sim = r3_sim(sc, pos, m, h, rho, precision, background)
    ref = oracle.pair_field_r3(pos, m, h, 1.0)
    if background == 3:
        ref += oracle.background_sphere(pos, 1.0, rho)
    med, _, mx = stats(sim.forces(), ref)
    assert med <= med_gate and mx <= max_gate
    sim.close()


@pytest.mark.parametrize("n", [2, 129, 1000])
def test_r3_ragged_sizes(sc, n):
    pos, m, h, rho = ball(n, 100 + n, R=1.0)
    sim = r3_sim(sc, pos, m, h, rho, 1, 0)
    med, _, mx = stats(sim.forces(), oracle.pair_field_r3(pos, m, h, 1.0))
    assert med <= 2e-6 and mx <= 1e-4
    sim.close()


def test_r3_comoving_kdk_matches_oracle(sc):
    pos, m, h, rho = ball(300, 3)
    vel = np.random.default_rng(4).normal(0.0, 0.05, pos.shape)
    c = oracle.make_cosmo()
    t0 = ics.lcdm_time_of_a(0.1)
    dt = 0.02 * t0
    xo, po, ao, to = oracle.kdk(pos, vel * 0.1 ** 2, m, h, 1.0, 1.0, 1, 2.0, rho, 3, c, 0.1, t0, dt, 6, topology=1)
    cfg = sc.Config(topology=sc.STEPS_TOPO_R3, n_cut=1, precision=0, background=sc.STEPS_BG_SPHERE, rho_bar=rho,
                    R_sim=2.0, comoving=True, a_start=0.1, t_start=t0)
    sim = sc.Simulation(cfg, pos, vel, m, h)
    sim.step(dt, 6)
    xg, vg, a, t = sim.state()
    assert a == pytest.approx(ao, rel=1e-14) and t == pytest.approx(to, rel=1e-14)
    assert np.abs(xg - xo).max() <= 1e-10 * np.abs(xo - pos).max()
    assert np.abs(vg - po / ao ** 2).max() <= 1e-10 * np.abs(po / ao ** 2).max()
    sim.close()


def test_topology_combinations_are_checked(sc):
    pos, m, h, rho = ball(200, 5)
    for kw in ({"background": sc.STEPS_BG_FINITE}, {"tail": sc.STEPS_TAIL_SURROGATE}):
        with pytest.raises(sc.StepsError) as e:
            r3_sim(sc, pos, m, h, rho, 1, kw.pop("background", 0), **kw)
        assert e.value.code == sc.STEPS_EINVAL
    sim = r3_sim(sc, pos, m, h, rho, 1, 0)
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_build_tail_table(sim.ctx, 33, 5)
    assert e.value.code == sc.STEPS_EINVAL
    sim.close()
    d = ics.particle_load(200, 5, 1.0)
    for cfg in (sc.Config(background=sc.STEPS_BG_SPHERE), sc.Config(G=0.0)):
        with pytest.raises(sc.StepsError) as e:
            sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
        assert e.value.code == sc.STEPS_EINVAL


def glass_load(n=500, seed=21):
    w = ics.WORKLOADS["lcdm_n65536"]
    return w, ics.particle_load(n, seed, w.M_tot, rho_bar=w.rho_bar)


def test_glass_making_matches_oracle(sc):
    # repulsive gravity (G = -1) in S1xR2 with the finite-cylinder term, comoving
    w, d = glass_load()
    c = oracle.make_cosmo()
    a0, t0 = 0.02, ics.lcdm_time_of_a(0.02)
    dt = 0.03 * t0
    xo, po, ao, to = oracle.kdk(d["pos"], np.zeros_like(d["pos"]), d["m"], d["h"], -1.0, 1.0, 16, ics.R_SIM,
                                w.rho_bar, 1, c, a0, t0, dt, 25)
    cfg = sc.Config(G=-1.0, n_cut=16, precision=0, rho_bar=w.rho_bar, comoving=True, a_start=a0, t_start=t0)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    sim.step(dt, 25)
    xg, vg, a, t = sim.state()
    dx = xg - xo
    dx[:, 2] -= np.round(dx[:, 2])
    assert np.abs(dx).max() <= 1e-9 * np.abs(xo - d["pos"]).max()
    sim.close()


def test_glass_making_settles(sc):
    # the RMS net comoving field of the repulsive run falls as the drag removes energy
    w, d = glass_load()
    a0, t0 = 0.02, ics.lcdm_time_of_a(0.02)
    cfg = sc.Config(G=-1.0, n_cut=16, precision=sc.STEPS_FP32_KAHAN, rho_bar=w.rho_bar, comoving=True, a_start=a0,
                    t_start=t0)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])

    def rms_field():
        _, _, a, _ = sim.state()
        g = sim.forces() * a ** 3
        return math.sqrt((g ** 2).sum(1).mean())

    r0, t = rms_field(), t0
    for _ in range(5):
        sim.step(0.03 * t, 25)
        t = sim.state()[3]
    r1 = rms_field()
    print(f"glass: RMS net field {r0:.3e} -> {r1:.3e} ({r1 / r0:.3f}), a = {sim.state()[2]:.3g}")
    assert r1 < 0.3 * r0
    sim.close()
