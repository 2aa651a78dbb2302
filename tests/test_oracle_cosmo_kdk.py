"""Pins of the oracle's background cosmology (eqs. Friedmann, DEdensity,
CPLw0wa; RK4, Sect. 2.3) and its KDK leapfrog (Sect. 2.1)."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2602_20787_gb300 import ics


def a_lcdm(t, Om=0.3, OL=0.7, H0=1.0):
    """Flat LCDM closed form a(t) = (Om/OL)^(1/3) sinh^(2/3)(1.5 sqrt(OL) H0 t)."""
    return (Om / OL) ** (1 / 3) * math.sinh(1.5 * math.sqrt(OL) * H0 * t) ** (2 / 3)


def test_hubble_flat_lcdm(orc):
    c = orc.make_cosmo()
    assert orc.hubble(c, 1.0) == pytest.approx(1.0, rel=1e-15)
    for a in (0.02, 0.1, 0.5, 2.0):
        assert orc.hubble(c, a) == pytest.approx(math.sqrt(0.3 / a ** 3 + 0.7), rel=1e-14)


def test_cpl_dark_energy_density(orc):
    # eq. DEdensity with eq. CPLw0wa, against numerical quadrature of the exponent
    c = orc.make_cosmo(H0=0.7, Omega_m=0.25, Omega_L=0.7, Omega_r=1e-4, w0=-0.9, wa=0.3)
    for a in (0.05, 0.3, 1.0, 1.5):
        expo, _ = integrate.quad(lambda ap: (1 + (-0.9 + 0.3 * (1 - ap))) / ap, 1.0, a, epsrel=1e-14)
        ode = 0.7 * math.exp(-3 * expo)
        ok = 1 - 0.25 - 1e-4 - 0.7
        ref = 0.7 * math.sqrt(1e-4 / a ** 4 + 0.25 / a ** 3 + ok / a ** 2 + ode)
        assert orc.hubble(c, a) == pytest.approx(ref, rel=1e-13)


def test_rk4_scale_factor_against_closed_form(orc):
    c = orc.make_cosmo()
    t0, dt = ics.run_schedule(ics.WORKLOADS["lcdm_n65536"])
    a = 0.02
    assert a_lcdm(t0) == pytest.approx(0.02, rel=1e-12)
    errs = []
    for nsub in (1, 2):
        a = 0.02
        for _ in range(200 * nsub):
            a = orc.a_step(c, a, dt / nsub)
        errs.append(abs(a - a_lcdm(t0 + 200 * dt)))
    assert a == pytest.approx(0.1, rel=1e-9)
    assert 10 < errs[0] / errs[1] < 22  # fourth order


def test_kdk_factors(orc):
    # K1 = Int dt/a over the first half step, K2 over the second, D = Int dt/a^2
    # over the step, integrated with a(t) by RK4: the local error of one step
    # is O(dt^5), so halving dt divides the error of a by ~32 and the relative
    # error of the O(dt) integrals by ~16.
    c = orc.make_cosmo()
    t0 = ics.lcdm_time_of_a(0.05)
    errs = []
    for dt in (1e-3, 5e-4):
        K1, D, K2, an = orc.kdk_factors(c, a_lcdm(t0), dt)
        rK1 = integrate.quad(lambda t: 1 / a_lcdm(t), t0, t0 + dt / 2, epsrel=1e-14)[0]
        rK2 = integrate.quad(lambda t: 1 / a_lcdm(t), t0 + dt / 2, t0 + dt, epsrel=1e-14)[0]
        rD = integrate.quad(lambda t: 1 / a_lcdm(t) ** 2, t0, t0 + dt, epsrel=1e-14)[0]
        e = [abs(K1 / rK1 - 1), abs(K2 / rK2 - 1), abs(D / rD - 1), abs(an / a_lcdm(t0 + dt) - 1)]
        assert max(e) < 3e-8
        errs.append(e)
    ratios = [e1 / e2 for e1, e2 in zip(*errs)]
    assert all(13 < r < 19 for r in ratios[:3])
    assert 24 < ratios[3] < 40
    s = orc.make_cosmo(comoving=False)
    assert orc.kdk_factors(s, 1.0, 0.01) == (0.005, 0.01, 0.005, 1.0)


def two_body(d=0.6, m=0.5):
    """Equal masses on a circular orbit in the x-y plane (same z: the image
    window is then fixed at 2 Ncut - 1 images, so the force is conservative)."""
    pos = np.array([[-d / 2, 0.0, 0.5], [d / 2, 0.0, 0.5]])
    return pos, np.array([m, m]), np.array([1e-3, 1e-3])


def image_potential(pos, m, n_cut):
    dR = np.linalg.norm(pos[0, :2] - pos[1, :2])
    ks = np.arange(-(n_cut - 1), n_cut)
    return -m[0] * m[1] * np.sum(1.0 / np.sqrt(dR * dR + ks * ks))


def circular_speed(orc, pos, m, h, n_cut):
    g = orc.pair_field(pos, m, h, 1.0, 1.0, n_cut)
    r = abs(pos[1, 0])
    return math.sqrt(abs(g[1, 0]) * r)


@pytest.mark.parametrize("dt", [0.02, 0.01])
def test_two_body_energy_bounded(orc, dt):
    n_cut = 4
    pos, m, h = two_body()
    v = circular_speed(orc, pos, m, h, n_cut)
    p = np.array([[0.0, -v, 0.0], [0.0, v, 0.0]])
    c = orc.make_cosmo(comoving=False)
    E0 = 0.5 * np.sum(m[:, None] * p * p) + image_potential(pos, m, n_cut)
    Es = []
    x, pp = pos, p
    for _ in range(40):
        x, pp, _, _ = orc.kdk(x, pp, m, h, 1.0, 1.0, n_cut, 1.0, 0.0, 0, c, 1.0, 0.0, dt, 25)
        Es.append(0.5 * np.sum(m[:, None] * pp * pp) + image_potential(x, m, n_cut))
    err = np.abs(np.array(Es) - E0) / abs(E0)
    assert err.max() < 5e-4 * (dt / 0.01) ** 2
    # no secular drift: second half no worse than the first half
    assert err[20:].max() < 1.5 * err[:20].max() + 1e-12


def test_kdk_second_order(orc):
    n_cut = 4
    pos, m, h = two_body()
    v = circular_speed(orc, pos, m, h, n_cut)
    p = np.array([[0.0, -v * 1.1, 0.0], [0.0, v * 1.1, 0.0]])
    c = orc.make_cosmo(comoving=False)
    T = 0.8
    res = []
    for ns in (20, 40, 80, 1280):
        x, _, _, _ = orc.kdk(pos, p, m, h, 1.0, 1.0, n_cut, 1.0, 0.0, 0, c, 1.0, 0.0, T / ns, ns)
        res.append(x)
    e1 = np.abs(res[0] - res[3]).max()
    e2 = np.abs(res[1] - res[3]).max()
    e3 = np.abs(res[2] - res[3]).max()
    assert 3.3 < e1 / e2 < 4.7 and 3.3 < e2 / e3 < 4.7


def test_kdk_time_reversible(orc):
    d = ics.particle_load(24, 3, 1.0)
    c = orc.make_cosmo(comoving=False)
    p0 = np.random.default_rng(1).normal(0, 0.05, (24, 3))
    x1, p1, _, _ = orc.kdk(d["pos"], p0, d["m"], d["h"], 1.0, 1.0, 8, ics.R_SIM, 0.0, 0, c, 1.0, 0.0, 1e-3, 30)
    x2, p2, _, _ = orc.kdk(x1, -p1, d["m"], d["h"], 1.0, 1.0, 8, ics.R_SIM, 0.0, 0, c, 1.0, 0.0, 1e-3, 30)
    dz = np.mod(x2[:, 2] - d["pos"][:, 2] + 0.5, 1.0) - 0.5
    np.testing.assert_allclose(x2[:, :2], d["pos"][:, :2], atol=1e-12)
    np.testing.assert_allclose(dz, 0.0, atol=1e-12)
    np.testing.assert_allclose(-p2, p0, atol=1e-12)


@pytest.mark.parametrize("comoving", [False, True])
def test_kdk_conserves_pz_and_lz(orc, comoving):
    # Sect. 1: P_z and L_z are conserved in S1xR2 (Noether); the background is radial
    w = ics.WORKLOADS["lcdm_n65536"]
    d = ics.particle_load(40, 8, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    c = orc.make_cosmo(comoving=comoving)
    p0 = np.random.default_rng(2).normal(0, 0.02, (40, 3))
    a0, t0 = (0.05, ics.lcdm_time_of_a(0.05)) if comoving else (1.0, 0.0)
    x, p, a1, t1 = orc.kdk(d["pos"], p0, d["m"], d["h"], 1.0, 1.0, 8, ics.R_SIM, w.rho_bar, 1, c, a0, t0, 1e-3, 12)
    m = d["m"]
    Pz0, Pz1 = np.sum(m * p0[:, 2]), np.sum(m * p[:, 2])
    Lz0 = np.sum(m * (d["pos"][:, 0] * p0[:, 1] - d["pos"][:, 1] * p0[:, 0]))
    Lz1 = np.sum(m * (x[:, 0] * p[:, 1] - x[:, 1] * p[:, 0]))
    scale = np.sum(m[:, None] * np.abs(p))
    assert abs(Pz1 - Pz0) < 1e-13 * scale
    assert abs(Lz1 - Lz0) < 1e-12 * scale
    assert t1 == pytest.approx(t0 + 12e-3)
    if comoving:
        assert a1 > a0


def test_free_particle_velocity_decays_as_a_minus_2(orc):
    # a single particle with background off feels no force: p = a^2 dx/dt is
    # constant and x advances by p Int dt / a^2
    c = orc.make_cosmo()
    t0 = ics.lcdm_time_of_a(0.02)
    pos = np.array([[0.5, 0.0, 0.25]])
    p0 = np.array([[1e-3, 0.0, 2e-3]])
    dt = 1e-4
    x, p, a1, t1 = orc.kdk(pos, p0, np.array([1.0]), np.array([0.1]), 1.0, 1.0, 4, 3.0, 0.0, 0, c, 0.02, t0, dt, 50)
    np.testing.assert_array_equal(p, p0)
    drift = integrate.quad(lambda t: 1 / a_lcdm(t) ** 2, t0, t0 + 50 * dt, epsrel=1e-13)[0]
    assert x[0, 0] == pytest.approx(0.5 + 1e-3 * drift, rel=1e-9)
