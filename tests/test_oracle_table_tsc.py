"""Pins of the oracle's triangular-shaped-cloud (TSC) read of the correction
table (Sect. 2.3: the table is read with CIC or TSC). With x in node units,
the nearest node i and d = x - i, the weights of nodes i - 1, i, i + 1 are
(1/2 - d)^2 / 2, 3/4 - d^2, (1/2 + d)^2 / 2 per axis. They sum to 1 and have
first moment d and second moment d^2 + 1/4 about node i, so the read
reproduces constants and linear functions exactly and turns x^2 into
x^2 + 1/4: the smoothing of a unit-width cloud. Nodes beyond the edge take the
edge value. The TSC table form converges to the exact windowed sum at second
order, like the bilinear read.

Also the paper's table over the nearest image alone (n0 = 0), which holds the
tail sums themselves: its nodes against brute-force image sums, and its
second-order convergence, far coarser than the residual table's at the same
grid."""
import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics

N_CUT, N0 = 64, 4
NX, NY, DR_MAX = 11, 9, 4.0


def tsc_cfg(nx=NX, ny=NY, dR_max=DR_MAX):
    return oracle.make_table_cfg(N_CUT, N0, nx, ny, dR_max, read=oracle.TABLE_TSC)


def table_of(f, nx=NX, ny=NY):
    """A table whose node (i, j) holds f(i, j) (node units) in both components
    (the second scaled by -2, to tell the components apart)."""
    tab = np.zeros((ny, nx, 2))
    for j in range(ny):
        for i in range(nx):
            tab[j, i] = (f(i, j), -2.0 * f(i, j))
    return tab


def read_nodes(tab, cfg, x, y):
    """The TSC read at node coordinates (x, y)."""
    return oracle.tail_table_read(tab, cfg, x / (cfg.nx - 1) * cfg.dR_max, 0.5 * y / (cfg.ny - 1))


def test_constant_everywhere_including_edges(orc):
    cfg = tsc_cfg()
    tab = table_of(lambda i, j: 3.25)
    rng = np.random.default_rng(1)
    pts = [(0.0, 0.0), (NX - 1.0, NY - 1.0), (0.2, NY - 1.3)] + [tuple(p) for p in rng.uniform(0, 1, (40, 2)) *
                                                                [NX - 1, NY - 1]]
    for x, y in pts:
        assert np.allclose(read_nodes(tab, cfg, x, y), (3.25, -6.5), rtol=1e-15)


def test_linear_reproduced_and_quadratic_shifted_by_a_quarter(orc):
    cfg = tsc_cfg()
    rng = np.random.default_rng(2)
    lin = table_of(lambda i, j: 1.5 - 0.7 * i + 2.0 * j)
    quad_x = table_of(lambda i, j: float(i * i))
    prod = table_of(lambda i, j: float(i * i) * float(j * j) + 0.5 * j)
    for _ in range(60):
        # interior: the three nodes of each axis lie inside the table
        x, y = rng.uniform(1.0, NX - 2.0), rng.uniform(1.0, NY - 2.0)
        assert read_nodes(lin, cfg, x, y)[0] == pytest.approx(1.5 - 0.7 * x + 2.0 * y, rel=1e-13)
        assert read_nodes(quad_x, cfg, x, y)[0] == pytest.approx(x * x + 0.25, rel=1e-13)
        r = read_nodes(prod, cfg, x, y)
        assert r[0] == pytest.approx((x * x + 0.25) * (y * y + 0.25) + 0.5 * y, rel=1e-13)
        assert r[1] == pytest.approx(-2.0 * r[0], rel=1e-15)


def test_at_a_node_and_at_the_edges(orc):
    cfg = tsc_cfg()
    f = lambda i, j: float(i) ** 3 + 0.1 * i   # varies along dR only
    tab = table_of(f)
    for i in (1, 4, NX - 2):
        # at a node: 3/4 of it and 1/8 of each neighbour
        want = 0.75 * f(i, 0) + 0.125 * (f(i - 1, 0) + f(i + 1, 0))
        assert read_nodes(tab, cfg, float(i), 3.0)[0] == pytest.approx(want, rel=1e-14)
    # the first node: its missing neighbour takes its own value
    assert read_nodes(tab, cfg, 0.0, 3.0)[0] == pytest.approx(0.875 * f(0, 0) + 0.125 * f(1, 0), abs=1e-15)
    # the last node, and dR beyond dR_max reads as the last node
    last = 0.875 * f(NX - 1, 0) + 0.125 * f(NX - 2, 0)
    assert read_nodes(tab, cfg, NX - 1.0, 3.0)[0] == pytest.approx(last, rel=1e-14)
    assert oracle.tail_table_read(tab, cfg, 3.0 * DR_MAX, 0.2)[0] == pytest.approx(last, rel=1e-14)
    # the nearest node switches at the half-way point without a jump
    lo = read_nodes(tab, cfg, 4.5 - 1e-9, 2.0)[0]
    hi = read_nodes(tab, cfg, 4.5 + 1e-9, 2.0)[0]
    assert lo == pytest.approx(hi, rel=1e-7)


def test_tsc_table_form_converges_to_the_windowed_sum(orc):
    w = ics.WORKLOADS["surrogate_n1048576"]
    d = ics.particle_load(1024, 3, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    idx = ics.subsample(1024, 48, seed=5)
    dR_max = 2.2 * np.hypot(d["pos"][:, 0], d["pos"][:, 1]).max()
    exact = oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, N_CUT, idx=idx)
    errs = []
    for nx, ny in [(65, 9), (129, 17), (257, 33)]:
        cfg = tsc_cfg(nx, ny, dR_max)
        tab = oracle.tail_table_build(cfg)
        g = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, tab, cfg, idx=idx)
        errs.append(np.median(np.linalg.norm(g - exact, axis=1) / np.linalg.norm(exact, axis=1)))
    print("TSC table form median errors:", errs)
    assert errs[-1] < 1e-7
    for a, b in zip(errs, errs[1:]):
        assert 2.5 < a / b < 6.5   # second order: halving the spacing divides the error by ~4


def test_nearest_image_table_holds_the_raw_tail(orc):
    # n0 = 0, the paper's D over the nearest image: no base, unit envelope, so a
    # node is the point-mass sum of every image but the nearest (brute force)
    for n_cut in (N_CUT, 0):
        cfg = oracle.make_table_cfg(n_cut, 0, 9, 5, 2.0)
        tab = oracle.tail_table_build(cfg)
        for i, j in [(0, 0), (3, 2), (8, 4), (5, 1)]:
            dR, adz = 2.0 * i / 8, 0.5 * j / 4
            kmax = n_cut + 1 if n_cut else 200000
            ks = np.array([k for k in range(-kmax, kmax + 1) if k != 0 and (n_cut == 0 or abs(adz + k) < n_cut)],
                          dtype=float)
            o = adz + ks
            r3 = (dR * dR + o * o) ** -1.5
            tol = 1e-12 if n_cut else 1e-9   # the brute-force line is cut at |k| = 2e5
            assert tab[j, i, 0] == pytest.approx(r3.sum(), rel=tol)
            assert tab[j, i, 1] == pytest.approx((o * r3).sum(), rel=tol, abs=1e-12)


def test_nearest_image_table_converges_at_second_order(orc):
    w = ics.WORKLOADS["surrogate_n1048576"]
    d = ics.particle_load(1024, 3, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    idx = ics.subsample(1024, 48, seed=5)
    dR_max = 2.2 * np.hypot(d["pos"][:, 0], d["pos"][:, 1]).max()
    exact = oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, N_CUT, idx=idx)
    errs = []
    for nx, ny in [(65, 9), (129, 17), (257, 33)]:
        cfg = oracle.make_table_cfg(N_CUT, 0, nx, ny, dR_max)
        g = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, oracle.tail_table_build(cfg), cfg, idx=idx)
        errs.append(np.median(np.linalg.norm(g - exact, axis=1) / np.linalg.norm(exact, axis=1)))
    print("nearest-image table median errors:", errs)
    assert 1e-5 < errs[-1] < 1e-4   # far coarser than the residual table at the same grid
    for a, b in zip(errs, errs[1:]):
        assert 2.5 < a / b < 6.5
