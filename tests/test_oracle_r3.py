"""Pins of the oracle's R^3 topology (Sect. 2.1, eq. NewtonianForce: the
softened Newtonian pair force without images, and the radial term
+(4 pi G / 3) rho0 x of a comoving homogeneous ball) and of its KDK."""
import math

import numpy as np
import pytest

import oracle


def test_two_body_closed_form(orc):
    pos = np.array([[0.1, -0.2, 0.3], [0.1 + 2.0, -0.2, 0.3 + 1.5]])   # |r| = 2.5
    m = np.array([1.5, 0.5])
    h = np.array([0.3, 0.4])                                             # h_i + h_j = 0.7 < 2.5: Newtonian
    g = oracle.pair_field_r3(pos, m, h, 2.0)
    r = pos[0] - pos[1]
    assert np.allclose(g[0], -2.0 * m[1] * r / 2.5 ** 3, rtol=1e-14)
    assert np.allclose(g[1], 2.0 * m[0] * r / 2.5 ** 3, rtol=1e-14)
    # inside the support the spline softens the force; at r -> 0 F/r -> 32 / (3 H^3)
    pos2 = np.array([[0.0, 0.0, 0.0], [1e-7, 0.0, 0.0]])
    g2 = oracle.pair_field_r3(pos2, np.array([1.0, 1.0]), np.array([0.5, 0.5]), 1.0)
    assert g2[0, 0] == pytest.approx(32.0 / 3.0 * 1e-7, rel=1e-6)


def test_newton_third_law_and_invariance(orc):
    rng = np.random.default_rng(5)
    n = 300
    pos = rng.normal(0.0, 1.0, (n, 3))
    m = rng.uniform(0.5, 2.0, n)
    h = rng.uniform(0.05, 0.4, n)
    g = oracle.pair_field_r3(pos, m, h, 1.0)
    assert np.abs((m[:, None] * g).sum(0)).max() <= 1e-12 * np.abs(m[:, None] * g).sum()
    # a rotation and a translation of the load rotate the field
    th = 0.7
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(1.1), -math.sin(1.1)], [0, math.sin(1.1), math.cos(1.1)]])
    Q = Rx @ Rz
    g2 = oracle.pair_field_r3(pos @ Q.T + np.array([3.0, -1.0, 2.0]), m, h, 1.0)
    assert np.allclose(g2, g @ Q.T, rtol=1e-10, atol=1e-12 * np.abs(g).max())


def test_point_symmetric_load_has_no_force_at_its_centre(orc):
    rng = np.random.default_rng(6)
    half = rng.normal(0.0, 1.0, (200, 3))
    pos = np.concatenate([np.zeros((1, 3)), half, -half])
    m = np.concatenate([[1.0], rng.uniform(0.5, 2.0, 200)])
    m = np.concatenate([m, m[1:]])
    h = np.full(401, 0.1)
    g = oracle.pair_field_r3(pos, m, h, 1.0, idx=np.array([0]))
    assert np.abs(g).max() <= 1e-13


def test_uniform_ball_and_radial_term_cancel(orc):
    # shell theorem: inside a homogeneous ball the pair field is -(4 pi G / 3) rho x,
    # which the radial term +(4 pi G / 3) rho x cancels. The ball is a cubic lattice
    # (no sampling noise), softened over two spacings; rho is mass per lattice cell.
    s = 0.05
    g1 = np.arange(-1.0, 1.0 + 1e-9, s) + s / 2
    X, Y, Z = np.meshgrid(g1, g1, g1, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pos = pos[np.linalg.norm(pos, axis=1) < 1.0]
    n = len(pos)
    m = np.full(n, 1.0 / n)
    rho = (1.0 / n) / s ** 3
    for probe in ([0.3, 0.2, -0.25], [-0.1, 0.35, 0.1]):
        probe = np.array([probe])
        load = np.concatenate([probe, pos])
        g = oracle.pair_field_r3(load, np.concatenate([[1e-12], m]), np.concatenate([[0.0], np.full(n, 2 * s)]), 1.0,
                                 idx=np.array([0]))[0]
        b = oracle.background_sphere(probe, 1.0, rho)[0]
        assert np.allclose(b, 4.0 * math.pi * rho / 3.0 * probe[0], rtol=1e-15)
        assert np.linalg.norm(g + b) < 2e-3 * np.linalg.norm(b)


def test_r3_kdk_keeps_a_circular_orbit(orc):
    # two equal masses on a circular orbit in static space, R^3, no background
    G, M, d = 1.0, 1.0, 1.0                  # separation d, each mass M
    v = math.sqrt(G * M / (2.0 * d))        # circular speed of each body about the centre
    pos = np.array([[0.5 * d, 0.0, 0.0], [-0.5 * d, 0.0, 0.0]])
    vel = np.array([[0.0, v, 0.0], [0.0, -v, 0.0]])
    period = 2.0 * math.pi * (0.5 * d) / v
    c = oracle.make_cosmo(comoving=False)
    steps = 4000
    x, p, a, t = oracle.kdk(pos, vel, np.array([M, M]), np.array([1e-4, 1e-4]), G, 1.0, 1, 1.0, 0.0, 0, c, 1.0,
                            0.0, period / steps, steps, topology=1)
    assert t == pytest.approx(period, rel=1e-12)
    assert np.allclose(x, pos, atol=2e-4)    # back where it started after one period
    sep = np.linalg.norm(x[0] - x[1])
    assert sep == pytest.approx(d, rel=1e-5)
