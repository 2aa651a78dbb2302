"""Pins of the oracle's diagnostics (Sect. 1: P_z and L_z are the conserved
quantities of S1xR2; the kinetic energy and the total mass are plain sums).

The oracle's or_diagnostics is checked against values worked out by hand for
three particles, against the transformation laws of momentum and angular
momentum under rotations and translations, and against the conservation of P_z
and L_z by the oracle's own KDK (translation along the axis and rotation about
it leave the S1xR2 force law invariant, so Noether's theorem conserves them).
A dropped a^2, a sign flip in L_z or a swapped component fails one of them."""
import numpy as np
import pytest

from paper_2602_20787_gb300 import ics


def three_particles():
    pos = np.array([[1.0, 0.0, 0.1], [0.0, 2.0, 0.5], [-1.0, -1.0, 0.9]])
    p = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 2.0], [2.0, -1.0, 0.0]])
    m = np.array([1.0, 2.0, 3.0])
    return pos, p, m


def test_hand_computed_three_particles(orc):
    pos, p, m = three_particles()
    d = orc.diagnostics(pos, p, m, 2.0)
    # P = 1 (0, 1, 0) + 2 (1, 0, 2) + 3 (2, -1, 0) = (8, -2, 4)
    assert d[0] == 8.0 and d[1] == -2.0 and d[2] == 4.0
    # L_z: 1 (1*1 - 0*0) + 2 (0*0 - 2*1) + 3 ((-1)(-1) - (-1)(2)) = 1 - 4 + 9 = 6
    assert d[3] == 6.0
    # |p|^2 = 1, 5, 5; sum m |p|^2 = 1 + 10 + 15 = 26; K = 26 / (2 a^4) = 13 / 16 at a = 2
    assert d[4] == 0.8125
    assert d[5] == 6.0


def test_static_kinetic_energy_of_one_particle(orc):
    # a = 1: dx/dt = p; m = 2, |v| = 5 gives K = 25
    d = orc.diagnostics(np.array([[0.3, -0.2, 0.4]]), np.array([[3.0, 4.0, 0.0]]), np.array([2.0]), 1.0)
    assert d[4] == 25.0 and d[5] == 2.0


def test_transformation_laws(orc):
    rng = np.random.default_rng(7)
    n = 200
    pos = rng.uniform(-2.0, 2.0, (n, 3))
    p = rng.normal(0.0, 1.0, (n, 3))
    m = rng.uniform(0.5, 2.0, n)
    a = 0.37
    d0 = orc.diagnostics(pos, p, m, a)
    # rotation about z by phi: P_xy rotates, P_z, L_z, K and the mass stay
    phi = 0.731
    c, s = np.cos(phi), np.sin(phi)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    d1 = orc.diagnostics(pos @ R.T, p @ R.T, m, a)
    np.testing.assert_allclose(d1[:3], R @ d0[:3], rtol=0, atol=1e-12 * np.abs(d0[:3]).max())
    np.testing.assert_allclose(d1[3:], d0[3:], rtol=1e-13)
    # translation by (dx, dy, dz): L_z -> L_z + dx P_y - dy P_x, the rest unchanged
    dx, dy, dz = 0.4, -1.3, 0.25
    d2 = orc.diagnostics(pos + np.array([dx, dy, dz]), p, m, a)
    np.testing.assert_allclose(d2[3], d0[3] + dx * d0[1] - dy * d0[0], rtol=1e-13)
    np.testing.assert_array_equal(d2[[0, 1, 2, 4, 5]], d0[[0, 1, 2, 4, 5]])
    # kinetic energy scales as a^-4 at fixed canonical momenta
    d3 = orc.diagnostics(pos, p, m, 2.0 * a)
    assert d3[4] == pytest.approx(d0[4] / 16.0, rel=1e-14)


def test_pz_and_lz_conserved_by_the_oracle_kdk(orc):
    w = ics.WORKLOADS["lcdm_n65536"]
    n, steps = 96, 8
    d = ics.particle_load(n, 5, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    vel = np.random.default_rng(3).normal(0.0, 0.05, (n, 3))
    t0, dt = ics.run_schedule(w)
    c = orc.make_cosmo()
    p0 = vel * w.a_start ** 2
    d0 = orc.diagnostics(d["pos"], p0, d["m"], w.a_start)
    x1, p1, a1, _ = orc.kdk(d["pos"], p0, d["m"], d["h"], 1.0, 1.0, 4, ics.R_SIM, w.rho_bar, 1, c, w.a_start, t0,
                            20 * dt, steps)
    d1 = orc.diagnostics(x1, p1, d["m"], a1)
    pscale = np.sum(d["m"][:, None] * np.abs(p1))
    lscale = np.sum(d["m"] * np.hypot(x1[:, 0], x1[:, 1]) * np.linalg.norm(p1, axis=1))
    assert abs(d1[2] - d0[2]) <= 1e-13 * pscale
    assert abs(d1[3] - d0[3]) <= 1e-13 * lscale
    # the radial background pushes P_x, P_y: they are not conserved, so the check above is not vacuous
    assert abs(d1[0] - d0[0]) > 1e-6 * pscale or abs(d1[1] - d0[1]) > 1e-6 * pscale
    assert d1[5] == pytest.approx(w.M_tot, rel=1e-14)
