"""Pins of the oracle's infinite window (Ncut -> infinity, Sect. 2.2): the whole
image line against the Fourier-Bessel closed form, the infinite base against
the finite one, the finite window's convergence to it, and the correction-table
form with the infinite window."""
import math

import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics
from tests.test_oracle_images import fourier_bessel_line


@pytest.mark.parametrize("dR,dz", [(0.3, 0.1), (0.7, -0.45), (1.0, 0.0), (1.9, 0.37), (0.15, -0.2), (5.0, 0.3)])
def test_infinite_line_matches_fourier_bessel(orc, dR, dz):
    sr, sz = oracle.image_sums_inf(dR, dz, 1e-9)
    FR, Fz = fourier_bessel_line(dR, dz)
    assert -dR * sr == pytest.approx(FR, rel=1e-11)
    assert -sz == pytest.approx(Fz, rel=1e-9, abs=1e-12)


def test_infinite_base_is_the_limit_of_the_finite_base(orc):
    for dR, adz in [(0.0, 0.2), (0.4, 0.0), (2.5, 0.45), (7.0, 0.1)]:
        bi = np.array(oracle.tail_base_inf(dR, adz, 4))
        bf = np.array(oracle.tail_base(dR, adz, 200000, 4))
        assert np.allclose(bi, bf, rtol=1e-9, atol=1e-10)


def test_finite_window_converges_to_the_infinite_one(orc):
    w = ics.WORKLOADS["surrogate_n1048576"]
    d = ics.particle_load(400, 3, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    idx = ics.subsample(400, 24, seed=1)
    g_inf = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx)
    diffs = []
    for n_cut in (64, 256):
        g = oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, n_cut, idx=idx)
        diffs.append(np.median(np.linalg.norm(g - g_inf, axis=1) / np.linalg.norm(g_inf, axis=1)))
    print("finite-window differences:", diffs)
    assert diffs[1] < 1e-4
    assert 10.0 < diffs[0] / diffs[1] < 22.0       # the truncation falls off as Ncut^-2


def test_infinite_table_form_converges(orc):
    w = ics.WORKLOADS["surrogate_n1048576"]
    d = ics.particle_load(600, 3, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    idx = ics.subsample(600, 32, seed=5)
    dR_max = 2.2 * np.hypot(d["pos"][:, 0], d["pos"][:, 1]).max()
    exact = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx)
    errs = []
    for nx, ny in [(65, 9), (129, 17), (257, 33)]:
        cfg = oracle.make_table_cfg(0, 4, nx, ny, dR_max)
        g = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, oracle.tail_table_build(cfg), cfg, idx=idx)
        errs.append(np.median(np.linalg.norm(g - exact, axis=1) / np.linalg.norm(exact, axis=1)))
    print("infinite table form median errors:", errs)
    assert errs[-1] < 1e-8
    for a, b in zip(errs, errs[1:]):
        assert 2.5 < a / b < 6.5


def constant_net(oracle_mod, y0, y1):
    w = np.zeros(oracle_mod.MLP_NW)
    w[-2], w[-1] = y0, y1     # output biases: the network is the constant (y0, y1)
    return w


@pytest.mark.parametrize("h", [1e-9, 0.4, 6.5, 11.0])
def test_inf_surrogate_with_the_exact_residual_is_the_line(orc, h):
    # a network that outputs the exact residual at (dR, |dz|) turns the surrogate
    # form of the infinite window into the exact line beyond n0, whatever the
    # sign of dz and however many tail images sit inside the softening support
    for dR, dz in [(0.3, 0.21), (1.7, -0.37), (4.0, 0.5), (0.05, -0.02)]:
        r = oracle.tail_residual(dR, abs(dz), 0, 4)
        cfg = oracle.make_surr_cfg(0, 4, 8.0, (0.0, 0.0), (1.0, 1.0))
        s = oracle.tail_surrogate(dR, dz, h, constant_net(oracle, r[0], r[1]), cfg)
        e = oracle.image_sums_inf(dR, dz, h, 4)
        assert s[0] == pytest.approx(e[0], rel=1e-12)
        assert s[1] == pytest.approx(e[1], rel=1e-11, abs=1e-15)


def test_inf_surrogate_zero_network_is_the_infinite_base(orc):
    w = np.zeros(oracle.MLP_NW)
    cfg = oracle.make_surr_cfg(0, 4, 8.0)
    for dR, dz in [(0.5, 0.3), (3.0, -0.1)]:
        s = oracle.tail_surrogate(dR, dz, 0.2, w, cfg)
        b = oracle.tail_base_inf(dR, abs(dz), 4)
        assert s[0] == pytest.approx(b[0], rel=1e-15) and s[1] == pytest.approx(np.sign(dz) * b[1], rel=1e-15)


def test_inf_surrogate_pair_field_converges_to_the_line(orc):
    # the zero network leaves only the base's Euler-Maclaurin remainder: small,
    # and of one order in the envelope
    d = ics.particle_load(80, 4, 1.0)
    g_s = oracle.pair_field_surrogate(d["pos"], d["m"], d["h"], 1.0, 1.0, np.zeros(oracle.MLP_NW),
                                      oracle.make_surr_cfg(0, 4, 8.0))
    g_e = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0)
    r = np.linalg.norm(g_s - g_e, axis=1) / np.linalg.norm(g_e, axis=1)
    assert np.median(r) < 1e-4
