"""GPU tests of the infinite window's correction table built by the Ewald
summation of the line (Sect. 2.3, eqs. cylindricalEwaldSplit, EwaldRealSum,
EwaldRecSum, with the Fourier kernel read as the line's incomplete Bessel
integral): its nodes against the oracle's Ewald sums over the oracle's base
and envelope, against the direct construction (the report and the oracle's
table), the forces it gives against the exact infinite line, the split
parameter's freedom, and the refused arguments."""
import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics
from tests.gpu_helpers import stats, table_dR_max

pytestmark = pytest.mark.gpu

N0 = 4
NX, NY = 144, 128   # the paper's table grid


@pytest.fixture(scope="module")
def sc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20787_gb300 import steps_cyl
    steps_cyl.load()
    return steps_cyl


def inf_config(sc, rho_bar, **kw):
    base = dict(n_cut=0, n0=N0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_TABLE,
                background=sc.STEPS_BG_INFINITE, rho_bar=rho_bar)
    base.update(kw)
    return sc.Config(**base)


def background(pos, rho_bar):
    return oracle.background_field(pos, ics.R_SIM, 0.0, 1.0, rho_bar, mode=2)


@pytest.fixture(scope="module")
def ewsim(sc):
    w = ics.WORKLOADS["surrogate_n1048576"]
    d = ics.particle_load(2600, 71, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    sim = sc.Simulation(inf_config(sc, w.rho_bar), d["pos"], d["vel"], d["m"], d["h"])
    rep = sc.steps_cyl_build_tail_table_ewald(sim.ctx, NX, NY, 0.0, 1.0, 5, 12)
    yield w, d, sim, rep
    sim.close()


def oracle_ewald_node(dR, adz, alpha=1.0, nmax=5, mmax=12):
    sr, sz = oracle.ewald_tail(dR, adz, N0, alpha, nmax, mmax)
    br, bz = oracle.tail_base_inf(dR, adz, N0)
    er, ez = oracle.tail_envelope(dR, adz, N0)
    return (sr - br) / er, (sz - bz) / ez


def test_report_against_direct_construction(sc, ewsim):
    *_, rep = ewsim
    diff, scale, t_ewald, t_direct = rep
    print(f"Ewald vs direct nodes: max diff {diff:.2e} of max |node| {scale:.2e}; "
          f"build {t_ewald:.2f} ms (Ewald) vs {t_direct:.2f} ms (direct)")
    assert scale > 0 and diff <= 1e-8 * max(scale, 1.0), (diff, scale)
    assert t_ewald > 0 and t_direct > 0


def test_nodes_match_oracle_ewald(sc, ewsim):
    _, d, sim, _ = ewsim
    tab, dR_max = sc.steps_cyl_get_tail_table(sim.ctx)
    assert tab.shape == (NY, NX, 2)
    assert dR_max == pytest.approx(table_dR_max(d["pos"]), rel=1e-15)
    rng = np.random.default_rng(5)
    nodes = [(0, 0), (NX - 1, NY - 1), (0, NY - 1), (NX - 1, 0)]
    nodes += [(int(i), int(j)) for i, j in zip(rng.integers(0, NX, 40), rng.integers(0, NY, 40))]
    scale = np.abs(tab).max()
    for i, j in nodes:
        ref = oracle_ewald_node(dR_max * i / (NX - 1), 0.5 * j / (NY - 1))
        assert np.allclose(tab[j, i], ref, rtol=2e-7, atol=1e-9 * scale), (i, j, tab[j, i], ref)


def test_nodes_match_oracle_direct_table(sc, ewsim):
    _, _, sim, _ = ewsim
    tab, dR_max = sc.steps_cyl_get_tail_table(sim.ctx)
    ref = oracle.tail_table_build(oracle.make_table_cfg(0, N0, NX, NY, dR_max))
    assert np.allclose(tab, ref, rtol=2e-7, atol=1e-9 * np.abs(ref).max())


def test_forces_against_exact_infinite_line(sc, ewsim):
    w, d, sim, _ = ewsim
    idx = ics.subsample(d["m"].shape[0], 160, seed=13)
    exact = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx) + background(d["pos"][idx], w.rho_bar)
    med, p999, mx = stats(sim.forces()[idx], exact)
    print(f"Ewald-table forces vs exact line: median {med:.2e} p99.9 {p999:.2e} max {mx:.2e}")
    assert med <= 1e-5 and p999 <= 1e-3


def test_split_parameter_is_free(sc):
    # the Ewald split is exact for any alpha: tables at two split parameters,
    # each with enough terms (the real-space images reach alpha r > 6, the
    # modes k^2 / (4 alpha^2) > 40), agree to FP32 rounding
    w = ics.WORKLOADS["surrogate_n1048576"]
    d = ics.particle_load(300, 72, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    sim = sc.Simulation(inf_config(sc, w.rho_bar), d["pos"], d["vel"], d["m"], d["h"])
    tabs = []
    for alpha, nmax, mmax in ((0.7, 9, 10), (2.0, 5, 24)):
        rep = sc.steps_cyl_build_tail_table_ewald(sim.ctx, 65, 33, 0.0, alpha, nmax, mmax)
        assert rep[0] <= 1e-8 * max(rep[1], 1.0), (alpha, rep)
        tabs.append(sc.steps_cyl_get_tail_table(sim.ctx)[0])
    sim.close()
    assert np.allclose(tabs[0], tabs[1], rtol=2e-7, atol=1e-9 * np.abs(tabs[0]).max())


def test_refused_arguments(sc):
    w = ics.WORKLOADS["surrogate_n1048576"]
    d = ics.particle_load(200, 73, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    finite = sc.Simulation(sc.Config(n_cut=16, n0=N0, rho_bar=w.rho_bar), d["pos"], d["vel"], d["m"], d["h"])
    with pytest.raises(sc.StepsError):
        sc.steps_cyl_build_tail_table_ewald(finite.ctx, 65, 33)
    finite.close()
    sim = sc.Simulation(inf_config(sc, w.rho_bar), d["pos"], d["vel"], d["m"], d["h"])
    for kw in (dict(alpha=0.1), dict(alpha=9.0), dict(nmax=N0 - 1), dict(nmax=65), dict(mmax=-1), dict(mmax=65),
               dict(nx=1), dict(ny=2000), dict(dR_max=-1.0)):
        args = dict(nx=65, ny=33, dR_max=0.0, alpha=1.0, nmax=5, mmax=12)
        args.update(kw)
        with pytest.raises(sc.StepsError):
            sc.steps_cyl_build_tail_table_ewald(sim.ctx, **args)
    # the table built at init is still in use after the refusals
    idx = ics.subsample(200, 50, seed=1)
    exact = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx) + background(d["pos"][idx], w.rho_bar)
    med, _, _ = stats(sim.forces()[idx], exact)
    assert med <= 1e-5
    sim.close()
