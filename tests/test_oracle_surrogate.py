"""Pins of the oracle's surrogate definition (this project's learned far-image
tail; the paper has no such method): the continuum base against independent
quadrature, the base's remainder against the next Euler-Maclaurin term, the
symmetry in dz, and the exact correction of softened tail images."""
import math

import numpy as np
import pytest
from scipy import integrate

N_CUT, N0 = 64, 4
A = N0 + 0.5


def f_R(z, R):
    return (R * R + z * z) ** -1.5


def f_Z(z, R):
    return z * (R * R + z * z) ** -1.5


def deriv(f, z, R, order, h=1e-2):
    # central finite differences (4th-order accurate stencils)
    if order == 1:
        return (-f(z + 2 * h, R) + 8 * f(z + h, R) - 8 * f(z - h, R) + f(z - 2 * h, R)) / (12 * h)
    if order == 3:
        return (-f(z + 3 * h, R) + 8 * f(z + 2 * h, R) - 13 * f(z + h, R) + 13 * f(z - h, R) - 8 * f(z - 2 * h, R)
                + f(z - 3 * h, R)) / (8 * h ** 3)
    raise ValueError


def sides(adz):
    kpos, kneg = N_CUT - 1, (N_CUT if adz > 0 else N_CUT - 1)
    return [(A + adz, kpos + 0.5 + adz, 1.0), (A - adz, kneg + 0.5 - adz, -1.0)]


@pytest.mark.parametrize("R", [0.0, 0.01, 0.7, 2.5, 6.0])
@pytest.mark.parametrize("adz", [0.0, 0.13, 0.5])
def test_base_is_integral_plus_first_euler_maclaurin_term(orc, R, adz):
    BR, BZ = orc.tail_base(R, adz, N_CUT, N0)
    eR = eZ = 0.0
    for lo, hi, sg in sides(adz):
        eR += integrate.quad(f_R, lo, hi, args=(R,), epsabs=0, epsrel=1e-13)[0] - (
            deriv(f_R, hi, R, 1) - deriv(f_R, lo, R, 1)) / 24
        eZ += sg * (integrate.quad(f_Z, lo, hi, args=(R,), epsabs=0, epsrel=1e-13)[0] - (
            deriv(f_Z, hi, R, 1) - deriv(f_Z, lo, R, 1)) / 24)
    assert BR == pytest.approx(eR, rel=1e-9)
    assert BZ == pytest.approx(eZ, rel=1e-8, abs=1e-14)


@pytest.mark.parametrize("R", [0.0, 0.3, 1.5, 4.0])
@pytest.mark.parametrize("adz", [0.05, 0.31, 0.5])
def test_base_remainder_is_the_next_euler_maclaurin_term(orc, R, adz):
    # exact tail minus base = +(7/5760) [f'''(end) - f'''(start)] + O(f^(5))
    SR, SZ = orc.tail_sums(R, adz, 1e-6, 1.0, N_CUT, N0)
    BR, BZ = orc.tail_base(R, adz, N_CUT, N0)
    pR = pZ = 0.0
    for lo, hi, sg in sides(adz):
        pR += 7.0 / 5760.0 * (deriv(f_R, hi, R, 3) - deriv(f_R, lo, R, 3))
        pZ += sg * 7.0 / 5760.0 * (deriv(f_Z, hi, R, 3) - deriv(f_Z, lo, R, 3))
    assert SR - BR == pytest.approx(pR, rel=0.1)
    assert SZ - BZ == pytest.approx(pZ, rel=0.1, abs=1e-9)
    assert abs(SR - BR) < 5e-4 * SR


def test_envelope_and_inputs(orc):
    ER, EZ = orc.tail_envelope(1.5, 0.2, N0)
    e = 1 / (1.5 ** 2 + 4.7 ** 2)
    assert ER == pytest.approx(e ** 3, rel=1e-14) and EZ == pytest.approx(e ** 2.5, rel=1e-14)
    np.testing.assert_allclose(orc.surrogate_inputs(2.0, 0.25, 1.0, N0, 8.0), [-0.5, 0.0, 2 / 4.5 - 1], rtol=1e-14)
    np.testing.assert_allclose(orc.surrogate_inputs(12.0, 0.5, 9.0, N0, 8.0), [1.0, 1.0, 1.0], rtol=1e-14)


def random_net(orc, seed=0, scale=0.3):
    return np.random.default_rng(seed).normal(0.0, scale, orc.MLP_NW)


def test_surrogate_symmetry_in_dz(orc):
    w = random_net(orc)
    cfg = orc.make_surr_cfg(N_CUT, N0, 8.0, (0.01, -0.002), (0.05, 0.005))
    for R, dz in ((0.3, 0.2), (2.0, 0.5), (5.0, 0.01)):
        a = orc.tail_surrogate(R, dz, 0.5, w, cfg)
        b = orc.tail_surrogate(R, -dz, 0.5, w, cfg)
        assert a[0] == pytest.approx(b[0], rel=1e-15) and a[1] == pytest.approx(-b[1], rel=1e-15)
    assert orc.tail_surrogate(1.0, 0.0, 0.5, w, cfg)[1] == 0.0


def test_zero_network_is_the_base_and_residual_is_added_with_envelope(orc):
    w = np.zeros(orc.MLP_NW)
    cfg = orc.make_surr_cfg(N_CUT, N0, 8.0)
    for R, dz in ((0.5, 0.3), (3.0, -0.1)):
        s = orc.tail_surrogate(R, dz, 0.2, w, cfg)
        b = orc.tail_base(R, abs(dz), N_CUT, N0)
        assert s[0] == pytest.approx(b[0], rel=1e-15) and s[1] == pytest.approx(np.sign(dz) * b[1], rel=1e-15)
    # a network whose output is the constant (1, 2) adds (mu + sc) * envelope
    w[-2], w[-1] = 1.0, 2.0  # output biases
    cfg = orc.make_surr_cfg(N_CUT, N0, 8.0, (0.5, -1.0), (2.0, 3.0))
    s = orc.tail_surrogate(1.0, 0.25, 0.2, w, cfg)
    b = orc.tail_base(1.0, 0.25, N_CUT, N0)
    E = orc.tail_envelope(1.0, 0.25, N0)
    assert s[0] == pytest.approx(b[0] + E[0] * (1.0 * 2.0 + 0.5), rel=1e-14)
    assert s[1] == pytest.approx(b[1] + E[1] * (2.0 * 3.0 - 1.0), rel=1e-14)


@pytest.mark.parametrize("h", [4.0, 6.5, 12.0])
def test_softened_tail_images_are_exact(orc, h):
    # with the network off, the surrogate differs from the exact (softened)
    # tail only by the base's Newtonian remainder, whatever the softening
    w = np.zeros(orc.MLP_NW)
    cfg = orc.make_surr_cfg(N_CUT, N0, 8.0)
    for R, dz in ((0.4, 0.21), (2.0, -0.37)):
        soft = orc.tail_surrogate(R, dz, h, w, cfg)
        exact = orc.tail_sums(R, dz, h, 1.0, N_CUT, N0)
        newton = orc.tail_sums(R, dz, 1e-9, 1.0, N_CUT, N0)
        base = orc.tail_surrogate(R, dz, 1e-9, w, cfg)
        assert soft[0] - exact[0] == pytest.approx(base[0] - newton[0], rel=1e-6, abs=1e-14)
        assert soft[1] - exact[1] == pytest.approx(base[1] - newton[1], rel=1e-6, abs=1e-14)


def test_pair_field_surrogate_near_part_and_base_error(orc):
    from paper_2602_20787_gb300 import ics
    d = ics.particle_load(60, 4, 1.0)
    cfg = orc.make_surr_cfg(N_CUT, N0, 8.0)
    w = np.zeros(orc.MLP_NW)
    g_s = orc.pair_field_surrogate(d["pos"], d["m"], d["h"], 1.0, 1.0, w, cfg)
    g_e = orc.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, N_CUT)
    r = np.linalg.norm(g_s - g_e, axis=1) / np.linalg.norm(g_e, axis=1)
    assert np.median(r) < 1e-4
    # period scaling: lengths in units of L
    lam = 2.5
    g2 = orc.pair_field_surrogate(d["pos"] * lam, d["m"], d["h"] * lam, 1.0, lam, w, cfg)
    np.testing.assert_allclose(g2 * lam * lam, g_s, rtol=1e-12, atol=1e-14 * np.abs(g_s).max())
