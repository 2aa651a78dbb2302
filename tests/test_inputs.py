"""The synthetic input recipe (Sect. 3.1 geometry; the workload laws):
masses, density, softening laws, the filament and the displacements, checked on
the generator itself so that every workload is the one its description states."""
import math

import numpy as np
import pytest

from paper_2602_20787_gb300 import ics


def test_geometry_constants():
    # D_s = L/2 and w < 0.9 pi give R_sim = (L/2) tan(0.45 pi) (eq. omegatovarrho)
    assert ics.R_SIM == pytest.approx(0.5 * math.tan(0.45 * math.pi), rel=1e-15)
    assert ics.R_SIM == pytest.approx(3.1569, abs=1e-4)


def test_mass_law_gives_uniform_expected_density():
    d = ics.particle_load(400_000, 3, 1.0)
    assert d["m"].sum() == pytest.approx(1.0, rel=1e-12)
    rho = np.hypot(d["pos"][:, 0], d["pos"][:, 1])
    assert rho.max() < ics.R_SIM and np.all((d["pos"][:, 2] >= 0) & (d["pos"][:, 2] < 1.0))
    edges = ics.R_SIM * np.sqrt(np.linspace(0.0, 1.0, 9))        # equal-area annuli
    mass, _ = np.histogram(rho, bins=edges, weights=d["m"])
    np.testing.assert_allclose(mass, 1.0 / 8, rtol=0.05)
    # m is proportional to J(w) = tan(w/2) sec^2(w/2), the volume element of the compact radius
    w = 2.0 * np.arctan(rho / ics.D_S)
    J = np.tan(0.5 * w) / np.cos(0.5 * w) ** 2
    np.testing.assert_allclose(d["m"] / d["m"].sum(), J / J.sum(), rtol=1e-9)


def test_softening_laws():
    lit = ics.particle_load(5000, 1, 1.0)
    assert lit["h"].min() == pytest.approx(0.01)
    np.testing.assert_allclose(lit["h"], 0.01 * (lit["m"] / lit["m"].min()) ** (1 / 3), rtol=1e-12)
    r8 = ics.particle_load(5000, 1, 1.0, eps_law="ratio8")
    assert r8["h"].min() == pytest.approx(0.01) and r8["h"].max() == pytest.approx(0.08)
    assert np.all(np.diff(r8["h"][np.argsort(r8["m"])]) >= 0)  # monotone in mass
    with pytest.raises(ValueError):
        ics.particle_load(10, 1, 1.0, eps_law="other")


def test_headline_load_statistics():
    d = ics.workload_ics("lcdm_n65536")
    assert np.median(d["h"]) == pytest.approx(0.45, abs=0.01)
    rng = np.random.default_rng(0)
    i, j = rng.integers(0, 65536, 20000), rng.integers(0, 65536, 20000)
    dR = np.hypot(*(d["pos"][i, :2] - d["pos"][j, :2]).T)
    assert np.mean(dR < d["h"][i] + d["h"][j]) == pytest.approx(0.77, abs=0.02)


def test_filament_and_displacements():
    w = ics.WORKLOADS["precision_n262144"]
    n = 20000
    d = ics.particle_load(n, w.seed, w.M_tot, displaced=False, rho_bar=w.rho_bar, filament_frac=0.2)
    vals, counts = np.unique(d["m"], return_counts=True)
    assert counts.max() == round(0.2 * n)                      # the filament shares one mass
    assert d["m"].sum() == pytest.approx(w.M_tot, rel=1e-12)
    fil = d["m"] == vals[np.argmax(counts)]
    r = np.hypot(d["pos"][fil, 0], d["pos"][fil, 1])
    assert np.std(d["pos"][fil, 0]) == pytest.approx(0.05, rel=0.05)
    assert np.median(r) == pytest.approx(0.05 * math.sqrt(2 * math.log(2)), rel=0.05)
    a = ics.particle_load(n, 9, w.M_tot, rho_bar=w.rho_bar)
    b = ics.particle_load(n, 9, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    # sigma_i = 0.02 (m_i / rho_bar)^(1/3); the two loads share the draws before the displacement
    sig = 0.02 * (a["m"] / w.rho_bar) ** (1 / 3)
    dxy = (b["pos"][:, :2] - a["pos"][:, :2]) / sig[:, None]
    assert np.std(dxy) == pytest.approx(1.0, rel=0.03)


def test_workloads_are_seeded():
    a = ics.workload_ics("plain_small_n2048")
    b = ics.workload_ics("plain_small_n2048")
    np.testing.assert_array_equal(a["pos"], b["pos"])
    w = ics.WORKLOADS["lcdm_n65536"]
    assert w.M_tot == pytest.approx(3 * 0.3 / (8 * math.pi) * math.pi * ics.R_SIM ** 2, rel=1e-14)
