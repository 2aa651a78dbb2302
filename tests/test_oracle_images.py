"""Pins of the oracle's image sum (eq. ForceCylindrical) and pair field
(eq. ComovingEquationsOfMotionCylindrical, pair term)."""
import math

import numpy as np
import pytest
from scipy import special

from paper_2602_20787_gb300 import ics


def fourier_bessel_line(dR, dz, L=1.0, mmax=400):
    """Field of an infinite periodic line of unit masses (G = 1) at (0, 0, nL),
    from the standard Fourier-Bessel expansion of the lattice sum:
      F_R = -2/(L dR) - (4/L) sum_m k_m K1(k_m dR) cos(k_m dz)
      F_z =            - (4/L) sum_m k_m K0(k_m dR) sin(k_m dz),  k_m = 2 pi m / L."""
    k = 2 * math.pi * np.arange(1, mmax + 1) / L
    FR = -2.0 / (L * dR) - 4.0 / L * np.sum(k * special.k1(k * dR) * np.cos(k * dz))
    Fz = -4.0 / L * np.sum(k * special.k0(k * dR) * np.sin(k * dz))
    return FR, Fz


def window_remainder(dR, rz, n_cut, L=1.0):
    """Continuum integral of the images beyond the window |o| < n_cut L, on the
    cells of unit length around them (the error of this midpoint rule is
    O(f'(n_cut L)) ~ 1e-15 at n_cut = 4000)."""
    offs = np.array([rz - n * L for n in range(-n_cut, n_cut + 1) if abs(rz - n * L) < n_cut * L])
    top, bot = offs.max() + 0.5 * L, offs.min() - 0.5 * L
    # Int dR/(dR^2+o^2)^1.5 do = o/(dR sqrt(dR^2+o^2)); Int o/(...)^1.5 do = -1/sqrt(dR^2+o^2)
    s_top = 1.0 / dR - top / (dR * math.hypot(dR, top))
    s_bot = 1.0 / dR + bot / (dR * math.hypot(dR, bot))
    FR = -(s_top + s_bot) / L
    Fz = -(1.0 / math.hypot(dR, top) - 1.0 / math.hypot(dR, bot)) / L
    return FR, Fz


@pytest.mark.parametrize("dR,rz", [(0.3, 0.1), (0.7, -0.45), (1.0, 0.0), (1.9, 0.77), (0.15, -0.93), (5.0, 0.3)])
def test_converged_window_matches_fourier_bessel(orc, dR, rz):
    n_cut = 4000
    f, cnt = orc.image_force((dR, 0.0, rz), 1e-9, 1.0, n_cut)
    assert cnt == (2 * n_cut - 1 if rz == 0.0 else 2 * n_cut)
    rR, rZ = window_remainder(dR, rz, n_cut)
    FR, Fz = fourier_bessel_line(dR, rz)
    assert f[0] + rR == pytest.approx(FR, rel=1e-11, abs=1e-13)
    assert f[2] + rZ == pytest.approx(Fz, rel=1e-9, abs=2e-12)
    assert f[1] == 0.0


def test_far_field_line_mass(orc):
    # R >> L: the image line acts as a line mass, F_R -> -2 G m / (L R)
    for R in (5.0, 8.0):
        f, _ = orc.image_force((R, 0.0, 0.37), 1e-6, 1.0, 4000)
        rR, _ = window_remainder(R, 0.37, 4000)
        assert f[0] + rR == pytest.approx(-2.0 / R, rel=1e-12)


def test_window_counts_and_tie(orc):
    # 2 Ncut images for rz != 0, 2 Ncut - 1 at rz = 0 (strict inequality)
    for n_cut in (1, 2, 16, 64):
        for rz in (0.3, -0.3, 0.999, -0.999, 0.5, -0.5):
            assert orc.image_force((1.0, 0.0, rz), 0.01, 1.0, n_cut)[1] == 2 * n_cut
        assert orc.image_force((1.0, 0.0, 0.0), 0.01, 1.0, n_cut)[1] == 2 * n_cut - 1


def test_small_hand_sums(orc):
    # dR = 1, rz = 0, Ncut = 2: images n = -1, 0, 1 -> F_x = -(1 + 2 / 2^1.5)
    f, cnt = orc.image_force((1.0, 0.0, 0.0), 1e-6, 1.0, 2)
    assert cnt == 3
    assert f[0] == pytest.approx(-(1.0 + 1.0 / math.sqrt(2.0)), rel=1e-15)
    assert f[2] == 0.0
    # rz = 0.25, Ncut = 1: images n = 0 (dz = 0.25) and n = 1 (dz = -0.75)
    f, cnt = orc.image_force((1.0, 0.0, 0.25), 1e-6, 1.0, 1)
    assert cnt == 2
    r0, r1 = math.sqrt(1.0625), 1.25
    assert f[0] == pytest.approx(-(1 / r0 ** 3 + 1 / r1 ** 3), rel=1e-15)
    assert f[2] == pytest.approx(-(0.25 / r0 ** 3 - 0.75 / r1 ** 3), rel=1e-14)


def test_period_scaling(orc):
    # F(lambda r, L lambda, h lambda) = F(r, L, h) / lambda^2
    lam = 3.7
    f1, _ = orc.image_force((0.4, -0.2, 0.33), 0.5, 1.0, 16)
    f2, _ = orc.image_force((0.4 * lam, -0.2 * lam, 0.33 * lam), 0.5 * lam, lam, 16)
    np.testing.assert_allclose(f2 * lam * lam, f1, rtol=1e-13)


def test_anisotropy_against_r3(orc):
    # Sect. 2.1: S1xR2 force is stronger than R3 radially and weaker axially
    fr, _ = orc.image_force((0.3, 0.0, 0.0), 1e-6, 1.0, 64)
    assert -fr[0] > 1.0 / 0.3 ** 2
    fz, _ = orc.image_force((0.0, 0.0, 0.3), 1e-6, 1.0, 64)
    assert 0 < -fz[2] < 1.0 / 0.3 ** 2


def small_system(n, seed):
    d = ics.particle_load(n, seed, 1.0)
    return d["pos"], d["m"], d["h"]


def test_pair_field_is_sum_of_image_forces(orc):
    pos, m, h = small_system(7, 11)
    g = orc.pair_field(pos, m, h, 1.3, 1.0, 3)
    for i in range(7):
        s = np.zeros(3)
        for j in range(7):
            if j != i:
                f, _ = orc.image_force(pos[i] - pos[j], h[i] + h[j], 1.0, 3)
                s += 1.3 * m[j] * f
        np.testing.assert_allclose(g[i], s, rtol=1e-13, atol=1e-15)
    idx = np.array([5, 0, 3])
    np.testing.assert_allclose(orc.pair_field(pos, m, h, 1.3, 1.0, 3, idx=idx), g[idx], rtol=0, atol=0)


def test_newton_third_law(orc):
    pos, m, h = small_system(96, 5)
    g = orc.pair_field(pos, m, h, 1.0, 1.0, 16)
    net = (m[:, None] * g).sum(0)
    scale = (m[:, None] * np.abs(g)).sum()
    assert np.all(np.abs(net) < 1e-14 * scale)


def test_translation_and_rotation_invariance(orc):
    pos, m, h = small_system(48, 9)
    g0 = orc.pair_field(pos, m, h, 1.0, 1.0, 8)
    # translation along the periodic axis (z wraps into [0, L))
    p1 = pos.copy()
    p1[:, 2] = np.mod(p1[:, 2] + 0.6180339887, 1.0)
    np.testing.assert_allclose(orc.pair_field(p1, m, h, 1.0, 1.0, 8), g0, rtol=1e-10, atol=1e-12 * np.abs(g0).max())
    # translation in the x-y plane
    p2 = pos + np.array([1.7, -0.4, 0.0])
    np.testing.assert_allclose(orc.pair_field(p2, m, h, 1.0, 1.0, 8), g0, rtol=1e-10, atol=1e-12 * np.abs(g0).max())
    # rotation about z
    c, s = math.cos(0.9), math.sin(0.9)
    Rm = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    g3 = orc.pair_field(pos @ Rm.T, m, h, 1.0, 1.0, 8)
    np.testing.assert_allclose(g3, g0 @ Rm.T, rtol=1e-10, atol=1e-12 * np.abs(g0).max())


@pytest.mark.parametrize("rz", [0.37, -0.37, 0.0, 0.5, -0.5, 0.93, -0.01])
def test_tail_plus_near_is_the_window(orc, rz):
    # wrapped-frame window of the tail routine == the paper's window on raw r_z
    dR, h, n_cut, n0 = 0.8, 0.05, 16, 4
    f, _ = orc.image_force((dR, 0.0, rz), h, 1.0, n_cut)
    SR, Sz = orc.tail_sums(dR, rz - math.floor(rz + 0.5), h, 1.0, n_cut, -1)
    assert -f[0] / dR == pytest.approx(SR, rel=1e-14)
    assert -f[2] == pytest.approx(Sz, rel=1e-12, abs=1e-15)
    # near images (|k| <= n0 in the wrapped frame) + tail = window
    dzw = rz - math.floor(rz + 0.5)
    SRt, Szt = orc.tail_sums(dR, dzw, h, 1.0, n_cut, n0)
    near_R = sum(orc.spline_F_over_r(math.hypot(dR, dzw + k), h) for k in range(-n0, n0 + 1))
    near_z = sum((dzw + k) * orc.spline_F_over_r(math.hypot(dR, dzw + k), h) for k in range(-n0, n0 + 1))
    assert SRt + near_R == pytest.approx(SR, rel=1e-14)
    assert Szt + near_z == pytest.approx(Sz, rel=1e-12, abs=1e-15)


def test_coincident_particles_exert_no_force_on_each_other(orc):
    # two particles at one point: r = 0 in the centre image, the spline centre is finite
    # and the separation vector is zero, so the pair adds nothing; the other images pull
    # symmetrically in +-z and cancel
    pos = np.array([[0.4, -0.2, 0.3], [0.4, -0.2, 0.3]])
    g = orc.pair_field(pos, np.array([1.0, 2.0]), np.array([0.05, 0.07]), 1.0, 1.0, 8)
    assert np.abs(g).max() <= 1e-15     # the +-z images cancel up to rounding
    # with a third particle the coincident pair feels the same pull per unit mass
    pos3 = np.vstack([pos, [[1.1, 0.5, 0.8]]])
    g3 = orc.pair_field(pos3, np.array([1.0, 2.0, 0.5]), np.array([0.05, 0.05, 0.05]), 1.0, 1.0, 8)
    np.testing.assert_allclose(g3[0], g3[1], rtol=1e-14, atol=1e-14 * np.abs(g3).max())
