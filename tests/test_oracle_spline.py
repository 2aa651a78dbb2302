"""Pins of the oracle's softened force (eq. Force_spline_kernel) against things
the paper and the mathematics fix independently of the oracle's code."""
import math

import numpy as np
import pytest
from scipy import integrate


def m4_density(s, h):
    """Monaghan & Lattanzio (1985) M4 cubic-spline density with support radius h,
    normalised to unit mass: central value 8/(pi h^3). The paper states that its
    softening corresponds to this kernel (Sect. 2.1)."""
    u = s / h
    if u < 0.5:
        return 8.0 / (math.pi * h ** 3) * (1.0 - 6.0 * u * u + 6.0 * u ** 3)
    if u < 1.0:
        return 8.0 / (math.pi * h ** 3) * 2.0 * (1.0 - u) ** 3
    return 0.0


@pytest.mark.parametrize("h", [0.02, 0.3, 1.7])
@pytest.mark.parametrize("u", [0.05, 0.2, 0.4999, 0.5, 0.63, 0.9, 0.999, 1.0, 1.4, 3.0])
def test_spline_is_enclosed_mass_of_m4(orc, h, u):
    # Gauss's law: F(r) r^2 = enclosed mass fraction of the smoothing density.
    r = u * h
    enclosed, _ = integrate.quad(lambda s: 4 * math.pi * s * s * m4_density(s, h), 0.0, min(r, h),
                                 points=[0.5 * h] if r > 0.5 * h else None, epsabs=0, epsrel=1e-13)
    assert orc.spline_F(r, h) * r * r == pytest.approx(enclosed, rel=2e-12, abs=1e-15)


def test_m4_normalisation():
    total, _ = integrate.quad(lambda s: 4 * math.pi * s * s * m4_density(s, 0.7), 0, 0.7, points=[0.35])
    assert total == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("h", [0.01, 1.0, 5.0])
def test_spline_continuity_and_limits(orc, h):
    # values at the branch points: 76/30 / h^2 at h/2 and 1/h^2 at h
    lo = orc.spline_F(0.5 * h * (1 - 1e-12), h)
    hi = orc.spline_F(0.5 * h * (1 + 1e-12), h)
    assert lo == pytest.approx(38.0 / 15.0 / h ** 2, rel=1e-9)
    assert hi == pytest.approx(38.0 / 15.0 / h ** 2, rel=1e-9)
    assert orc.spline_F(h * (1 - 1e-13), h) == pytest.approx(1.0 / h ** 2, rel=1e-9)
    assert orc.spline_F(h, h) == 1.0 / h ** 2
    # F/r is finite at r = 0 with value 32/(3 h^3)
    assert orc.spline_F_over_r(0.0, h) == pytest.approx(32.0 / (3.0 * h ** 3), rel=1e-15)
    # Newtonian outside the support
    for r in (1.0001 * h, 2 * h, 10 * h):
        assert orc.spline_F(r, h) == pytest.approx(1.0 / r ** 2, rel=1e-15)


def test_F_over_r_consistent(orc):
    for h in (0.05, 1.3):
        for r in np.linspace(1e-3 * h, 2 * h, 57):
            assert orc.spline_F_over_r(r, h) == pytest.approx(orc.spline_F(r, h) / r, rel=1e-12)
