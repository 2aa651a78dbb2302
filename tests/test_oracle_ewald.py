"""Pins of the oracle's Ewald summation of the infinite periodic line (Sect.
2.3, eqs. cylindricalEwaldSplit, EwaldRealSum, EwaldRecSum and the m = 0 term,
with the Fourier kernel re-derived).

- A closed form: on the axis at dz = 0 the images k != 0 sum to 2 zeta(3).
- The Fourier-Bessel lattice sum of a periodic line of point masses (a standard
  result, evaluated here with scipy's K0 and K1), for the whole line.
- Independence of the split parameter: the split is exact for any alpha.
- The truncation the paper quotes: 5 real-space images and 12 modes reach far
  below single precision at a suitable alpha.
- The reading of eq. Bkernel: the printed kernel tends to 2 exp(-k rho) as alpha
  grows (the doubly periodic slab's kernel), while the line's kernel must tend to
  2 K0(k rho); the re-derived integral does."""
import math

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")


def fourier_bessel_line(dR, dz, terms=200):
    """SR, SZ of every image of a unit-period line (force -(dR SR, SZ)):
    F_R = -2/R - 4 sum k K1(k R) cos(k z), F_z = -4 sum k K0(k R) sin(k z), k = 2 pi m."""
    m = np.arange(1, terms + 1)
    k = 2 * np.pi * m
    fr = -2.0 / dR - 4.0 * np.sum(k * scipy_special.k1(k * dR) * np.cos(k * dz))
    fz = -4.0 * np.sum(k * scipy_special.k0(k * dR) * np.sin(k * dz))
    return -fr / dR, -fz


def test_axis_closed_form(orc):
    sr, sz = orc.ewald_tail(0.0, 0.0, 0, 1.5, 8, 40)
    zeta3 = 1.2020569031595942854
    assert sr == pytest.approx(2 * zeta3, rel=1e-13)
    assert sz == 0.0


@pytest.mark.parametrize("dR,dz", [(0.4, 0.1), (1.0, -0.3), (0.7, 0.45), (2.0, 0.25)])
def test_matches_fourier_bessel(orc, dR, dz):
    ref = fourier_bessel_line(dR, dz)
    for alpha in (1.0, 2.5):
        sr, sz = orc.ewald_tail(dR, dz, -1, alpha, 8, 40)  # n0 = -1: the whole line
        assert sr == pytest.approx(ref[0], rel=1e-12)
        assert sz == pytest.approx(ref[1], rel=1e-11, abs=1e-13)


def test_independent_of_the_split_parameter(orc):
    for dR, dz, n0 in [(0.2, 0.3, 1), (0.0, 0.49, 4), (1.3, -0.2, 2)]:
        vals = np.array([orc.ewald_tail(dR, dz, n0, a, 9, 60) for a in (0.8, 1.6, 3.0)])
        scale = np.abs(vals).max()
        assert np.abs(vals - vals[0]).max() <= 2e-12 * scale, vals


def test_paper_truncation_reaches_below_single_precision(orc):
    # n_max = 5 real-space images and m_max = 12 modes (the paper's medium setting)
    worst = 0.0
    for dR in (0.0, 0.3, 1.1, 3.0):
        for dz in (0.0, 0.2, 0.45):
            ref = orc.image_sums_inf(dR, dz, 0.0, 4)
            got = orc.ewald_tail(dR, dz, 4, 1.0, 5, 12)
            worst = max(worst, abs(got[0] - ref[0]) / abs(ref[0]))
            worst = max(worst, abs(got[1] - ref[1]) / max(abs(ref[1]), abs(ref[0])))
    assert worst < 1e-9, worst


def test_printed_kernel_is_the_slab_form():
    # eq. Bkernel as printed, at a large split parameter, against 2 exp(-k rho)
    # (slab) and 2 K0(k rho) (line); and the re-derived kernel's integral against 2 K0
    k, rho, alpha = 2 * math.pi, 0.3, 40.0
    erfc = scipy_special.erfc
    printed = (math.exp(k * rho) * erfc(k / (2 * alpha) + alpha * rho)
               + math.exp(-k * rho) * erfc(k / (2 * alpha) - alpha * rho))
    assert printed == pytest.approx(2 * math.exp(-k * rho), rel=1e-6)
    assert abs(printed - 2 * scipy_special.k0(k * rho)) > 0.1 * 2 * scipy_special.k0(k * rho)  # 15 % off
    from scipy.integrate import quad
    B, _ = quad(lambda s: math.exp(-rho * rho * math.exp(s) - k * k / (4 * math.exp(s))), math.log(k * k / 300),
                math.log(alpha * alpha), limit=200)
    assert B == pytest.approx(2 * scipy_special.k0(k * rho), rel=1e-10)
