"""Pins of the oracle's correction-table tail (Sect. 2.3, eq.
S1R2EwaldCorrectionTable, restated for the windowed sum beyond the near
images): node values are the exact tail, the read is bilinear, and the table
form converges to the exact windowed image sum at the order of bilinear
interpolation."""
import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics

N_CUT, N0 = 64, 4


def test_nodes_are_the_exact_tail(orc):
    cfg = oracle.make_table_cfg(N_CUT, N0, 9, 5, 6.0)
    tab = oracle.tail_table_build(cfg)
    for i, j in [(0, 0), (3, 2), (8, 4), (5, 1)]:
        dR, adz = 6.0 * i / 8, 0.5 * j / 4
        # the read reproduces the node value
        assert np.array_equal(oracle.tail_table_read(tab, cfg, dR, adz), tab[j, i])
        # and the table form there is the exact point-mass tail (brute-force sum)
        for sgn in (1.0, -1.0):
            dz = sgn * adz
            sr, sz = oracle.tail_table(dR, dz, 0.0, tab, cfg)
            ks = [k for k in range(-N_CUT - 1, N_CUT + 2) if abs(k) > N0 and abs(dz + k) < N_CUT]
            o = dz + np.array(ks, dtype=float)
            r3 = (dR * dR + o * o) ** -1.5
            assert sr == pytest.approx(r3.sum(), rel=1e-12)
            assert sz == pytest.approx((o * r3).sum(), rel=1e-10, abs=1e-16)


def test_read_is_bilinear(orc):
    # a table holding a bilinear function is read back exactly anywhere
    cfg = oracle.make_table_cfg(N_CUT, N0, 7, 4, 3.0)
    x = 3.0 * np.arange(7) / 6
    y = 0.5 * np.arange(4) / 3
    f = lambda a, b: (1.5 - 0.7 * a + 2.0 * b + 0.3 * a * b, -0.2 + a * b)
    tab = np.zeros((4, 7, 2))
    for j in range(4):
        for i in range(7):
            tab[j, i] = f(x[i], y[j])
    rng = np.random.default_rng(3)
    for _ in range(50):
        a, b = rng.uniform(0, 3.0), rng.uniform(0, 0.5)
        assert np.allclose(oracle.tail_table_read(tab, cfg, a, b), f(a, b), rtol=1e-13, atol=1e-14)
    # dR beyond dR_max reads the last column
    assert np.allclose(oracle.tail_table_read(tab, cfg, 10.0, 0.25), f(3.0, 0.25), rtol=1e-13)


def test_table_form_converges_to_the_windowed_sum(orc):
    w = ics.WORKLOADS["surrogate_n1048576"]
    d = ics.particle_load(1024, 3, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    idx = ics.subsample(1024, 48, seed=5)
    dR_max = 2.2 * np.hypot(d["pos"][:, 0], d["pos"][:, 1]).max()
    exact = oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, N_CUT, idx=idx)
    errs = []
    for nx, ny in [(65, 9), (129, 17), (257, 33)]:
        cfg = oracle.make_table_cfg(N_CUT, N0, nx, ny, dR_max)
        g = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, oracle.tail_table_build(cfg), cfg, idx=idx)
        errs.append(np.median(np.linalg.norm(g - exact, axis=1) / np.linalg.norm(exact, axis=1)))
    print("table form median errors:", errs)
    assert errs[-1] < 1e-8
    for a, b in zip(errs, errs[1:]):
        assert 2.5 < a / b < 6.5   # second order: halving the spacing divides the error by ~4


def test_softened_tail_images_are_exact(orc):
    # h large enough that tail images lie inside the support: the table form
    # adds F(r,h)/r - 1/r^3 for those, so it equals the softened exact tail
    cfg = oracle.make_table_cfg(N_CUT, N0, 257, 33, 8.0)
    tab = oracle.tail_table_build(cfg)
    for dR, dz, h in [(0.3, 0.2, 7.5), (1.2, -0.4, 9.0), (0.0, 0.1, 6.0)]:
        sr, sz = oracle.tail_table(dR, dz, h, tab, cfg)
        er, ez = oracle.tail_sums(dR, dz, h, 1.0, N_CUT, N0)
        assert sr == pytest.approx(er, rel=1e-7)
        assert sz == pytest.approx(ez, rel=1e-6, abs=1e-10)
