"""The tessellated particle load (arXiv 2602.20787, Sect. 3.1, eqs.
inversestereographic and omegatovarrho, Fig. 4), pinned to the values the paper
prints (tests/golden/compact_load_table1_fig4.txt) and to the invariants of the
construction: the cells tile the cylinder, the core has one mass, the outer
rings are uniform in the compact radius, and the expected density is uniform."""
import math
import pathlib

import numpy as np
import pytest

from paper_2602_20787_gb300 import ics

GOLDEN = pathlib.Path(__file__).parent / "golden" / "compact_load_table1_fig4.txt"

# Newton's constant in Mpc (km/s)^2 / M_sun (IAU nominal solar mass parameter
# over the parsec); it converts Table 1's H0 into a comoving mean density.
G_MPC_KMS2_MSUN = 4.30091e-9


def golden():
    vals = {}
    for line in GOLDEN.read_text().splitlines():
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("="))
            vals[k] = float(v)
    return vals


def test_core_radius_matches_fig4_caption():
    g = golden()
    r = ics.compact_rings(40, 8, 4, D_s=g["fig4_D_S_mpc"], R_sim=g["fig4_R_sim_mpc"],
                          omega_c=g["fig4_omega_c_rad"], L=g["fig4_L_z_mpc"])
    assert round(r.rho_c, 1) == g["fig4_rho_c_mpc"]
    # eq. inversestereographic inverts eq. omegatovarrho
    assert math.isclose(2.0 * math.atan(r.rho_c / g["fig4_D_S_mpc"]), g["fig4_omega_c_rad"], rel_tol=1e-14)
    d = ics.compact_load(40, 8, 4, 3, D_s=g["fig4_D_S_mpc"], R_sim=g["fig4_R_sim_mpc"],
                         omega_c=g["fig4_omega_c_rad"], L=g["fig4_L_z_mpc"])
    rho = np.hypot(d["pos"][:, 0], d["pos"][:, 1])
    core = rho < r.rho_c
    assert core.sum() == r.n_in * 8 * 4
    assert np.all(d["m"][core] == d["m"][core][0])
    assert np.all(d["m"][~core] > d["m"][core][0] * (1.0 - 0.5 / r.n_in))


@pytest.mark.parametrize("n_out", [300, 400, 600])
def test_mass_range_matches_table1(n_out):
    """Table 1's particle masses follow from its geometry, its cosmology and N_p
    alone: the mass of a cell depends on n_phi x n_z only through N_p."""
    g = golden()
    geom = dict(D_s=g["table1_D_S_mpc"], R_sim=g["table1_R_sim_mpc"], omega_c=g["table1_omega_c_rad"],
                L=g["table1_L_z_mpc"])
    r1 = ics.compact_rings(n_out, 1, 1, **geom)
    per_ring = int(round(g["table1_N_p"] / (r1.n_in + r1.n_out)))
    r = ics.compact_rings(n_out, per_ring, 1, **geom)
    assert abs(r.n / g["table1_N_p"] - 1.0) < 1e-3
    rho_bar = g["table1_Omega_m"] * 3.0 * g["table1_H0_km_s_mpc"] ** 2 / (8.0 * math.pi * G_MPC_KMS2_MSUN)
    m = rho_bar * r.cell_volume
    # printed to two significant figures
    assert 0.95e11 <= m.min() <= 1.05e11 and round(m.min(), -10) == g["table1_M_p_min_msun"]
    assert 1.55e13 <= m.max() <= 1.65e13 and round(m.max(), -12) == g["table1_M_p_max_msun"]


def test_cells_tile_the_cylinder():
    R, L, rho_bar = 2.0, 1.5, 0.37
    d = ics.compact_load(17, 11, 5, 8, D_s=0.4, R_sim=R, omega_c=1.2, L=L, rho_bar=rho_bar)
    r = d["rings"]
    assert d["pos"].shape == (r.n, 3) and r.n == (r.n_in + 17) * 11 * 5
    assert math.isclose(d["m"].sum(), rho_bar * math.pi * R * R * L, rel_tol=1e-12)
    assert math.isclose(r.s_edges[-1], R * R, rel_tol=1e-15) and r.s_edges[0] == 0.0
    assert np.all(np.diff(r.s_edges) > 0.0)
    # every particle sits in its own cell (ring-major, then sector, then slab)
    nr = r.n_in + r.n_out
    ring = np.repeat(np.arange(nr), 11 * 5)
    sec = np.tile(np.repeat(np.arange(11), 5), nr)
    slab = np.tile(np.arange(5), nr * 11)
    s = d["pos"][:, 0] ** 2 + d["pos"][:, 1] ** 2
    tol = 1e-12 * R * R
    assert np.all(s >= r.s_edges[ring] - tol) and np.all(s <= r.s_edges[ring + 1] + tol)
    assert np.all(np.sqrt(s) < R)
    phi = np.mod(np.arctan2(d["pos"][:, 1], d["pos"][:, 0]), 2.0 * math.pi)
    dphi = 2.0 * math.pi / 11
    assert np.all(phi >= sec * dphi - 1e-12) and np.all(phi <= (sec + 1) * dphi + 1e-12)
    z = d["pos"][:, 2]
    assert np.all((z >= 0.0) & (z < L))
    assert np.all(z >= slab * (L / 5) - 1e-12) and np.all(z <= (slab + 1) * (L / 5) + 1e-12)
    # m_i = rho_bar V_i with V_i the exact cell volume
    v = 0.5 * (r.s_edges[ring + 1] - r.s_edges[ring]) * dphi * (L / 5)
    np.testing.assert_allclose(d["m"], rho_bar * v, rtol=1e-14)


def test_outer_rings_uniform_in_omega_and_core_continuous():
    D, R, wc = 0.3, 3.0, 0.9
    r = ics.compact_rings(25, 4, 4, D_s=D, R_sim=R, omega_c=wc)
    w = 2.0 * np.arctan(np.sqrt(r.s_edges[r.n_in:]) / D)
    assert math.isclose(w[0], wc, rel_tol=1e-14) and math.isclose(w[-1], r.omega_max, rel_tol=1e-14)
    np.testing.assert_allclose(np.diff(w), (r.omega_max - wc) / 25, rtol=1e-9)
    v = r.cell_volume
    assert np.all(v[: r.n_in] == v[0])
    assert np.all(np.diff(v[r.n_in:]) > 0.0)
    # the core cell matches the first outer cell up to the rounding of n_in
    assert abs(v[0] / v[r.n_in] - 1.0) <= 0.5 / r.n_in + 1e-12
    # thin outer rings: the volume ratio of the last to the first outer ring is the
    # ratio of the volume element rho d(rho) = (D^2 / 2) tan(w/2) sec^2(w/2) dw at
    # the ring midpoints (midpoint rule, error O(dw^2))
    fine = ics.compact_rings(4000, 1, 1, D_s=D, R_sim=R, omega_c=wc)
    J = lambda x: math.tan(0.5 * x) / math.cos(0.5 * x) ** 2
    vf = fine.cell_volume
    dw = (fine.omega_max - wc) / 4000
    assert math.isclose(vf[-1] / vf[fine.n_in], J(fine.omega_max - 0.5 * dw) / J(wc + 0.5 * dw), rel_tol=1e-5)


def test_without_core_is_the_plain_compact_grid():
    r = ics.compact_rings(30, 6, 2)
    assert r.n_in == 0 and r.rho_c == 0.0 and r.s_edges[0] == 0.0
    assert math.isclose(r.s_edges[-1], ics.R_SIM ** 2, rel_tol=1e-15)
    w = 2.0 * np.arctan(np.sqrt(r.s_edges) / ics.D_S)
    np.testing.assert_allclose(np.diff(w), ics.W_MAX / 30, rtol=1e-9)


def test_expected_density_is_uniform():
    """Mass in annuli that cut across the rings matches rho_bar times their volume
    (each particle is uniform in its cell, so the expected density is rho_bar)."""
    R, L = 1.0, 1.0
    d = ics.compact_load(160, 64, 16, 11, D_s=0.14, R_sim=R, omega_c=1.63973, L=L, rho_bar=1.0)
    rho = np.hypot(d["pos"][:, 0], d["pos"][:, 1])
    # annuli a few rings wide everywhere (the outer rings are ~0.03 R wide at the edge)
    edges = np.linspace(0.0, R, 11) ** 0.8
    mass, _ = np.histogram(rho, bins=edges, weights=d["m"])
    vol = math.pi * np.diff(edges ** 2) * L
    np.testing.assert_allclose(mass / vol, 1.0, rtol=0.03)
    # a random half-space through the axis holds half the mass
    frac = d["m"][d["pos"][:, 0] * 0.6 + d["pos"][:, 1] * 0.8 > 0.0].sum() / d["m"].sum()
    assert abs(frac - 0.5) < 0.01


def test_seeded_and_deterministic():
    a = ics.compact_load(12, 6, 3, 5, omega_c=1.0)
    b = ics.compact_load(12, 6, 3, 5, omega_c=1.0)
    c = ics.compact_load(12, 6, 3, 6, omega_c=1.0)
    np.testing.assert_array_equal(a["pos"], b["pos"])
    np.testing.assert_array_equal(a["m"], c["m"])
    assert not np.array_equal(a["pos"], c["pos"])
    assert a["h"].min() == 0.01 and math.isclose(a["h"].max(), 0.01 * (a["m"].max() / a["m"].min()) ** (1 / 3))


@pytest.mark.parametrize("kw", [dict(n_out=0), dict(n_phi=0), dict(omega_c=-0.1), dict(omega_c=3.2),
                                dict(D_s=0.0), dict(L=-1.0)])
def test_invalid_arguments(kw):
    args = dict(n_out=4, n_phi=4, n_z=4)
    args.update(kw)
    with pytest.raises(ValueError):
        ics.compact_rings(args.pop("n_out"), args.pop("n_phi"), args.pop("n_z"), **args)
