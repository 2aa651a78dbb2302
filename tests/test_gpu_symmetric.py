"""GPU parity of the symmetric pair kernels (pair_sym.cuh): each unordered pair
is evaluated once and added to both particles (Newton's third law, exact for
the symmetric window of eq. ForceCylindrical), into deterministic fixed-point
accumulators.

- Every FP32 direct form (plain Kahan and plain sums, correction table, learned
  tail, infinite window) against the row kernels, which evaluate each ordered
  pair (two emulated shards), and against the FP64 oracle.
- The modelled tails' straight-run kernels (near range n0 = 4, every h_i + h_j
  below L / 2, softened steps redone with the spline tiers) against the row
  kernels and the oracle's surrogate form.
- Newton's third law to the rounding of the FP32 partial sums.
- A softening so small that the fixed-point unit would be too coarse falls back
  to the row kernels."""
import numpy as np
import pytest

import oracle
from gpu_helpers import oracle_accel, rel_err, seeded_surrogate, stats
from paper_2602_20787_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20787_gb300 import shard, steps_cyl
    steps_cyl.load()
    return torch, steps_cyl, shard


def row_forces(sc, shard, cfg, d, setup=None):
    """The same forces from the row kernels: two emulated shards, summed."""
    out = 0.0
    for r in range(2):
        sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
        if setup:
            setup(sim)
        shard.GpuRows(sim, r, 2)
        out = out + sim.forces()
        assert not sc.steps_cyl_last_eval(sim.ctx)["symmetric"]
        sim.close()
    return out


def test_plain_forms_match_row_kernels_and_oracle(env):
    torch, sc, shard = env
    n = 2500   # 20 blocks, the last one ragged
    d = ics.particle_load(n, 61, 1.0)
    ref = oracle_accel(d["pos"], d["m"], d["h"], 16)
    for precision, med_gate in ((sc.STEPS_FP32_KAHAN, 1e-6), (sc.STEPS_FP32_PLAIN, 1e-5)):
        cfg = sc.Config(n_cut=16, precision=precision, reorder_every=-1)
        sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
        a = sim.forces()
        ev = sc.steps_cyl_last_eval(sim.ctx)
        assert ev["symmetric"]
        # each unordered pair once, the pairs inside a 128-row block both ways
        within = sum(k * (k - 1) for k in [128] * 19 + [n - 19 * 128])
        assert ev["pairs_evaluated"] == pytest.approx((n * (n - 1) - within) / 2 + within, rel=1e-15)
        assert ev["pair_images"] == n * (n - 1) * 32
        sim.close()
        rows = row_forces(sc, shard, cfg, d)
        r = rel_err(a, rows)
        assert np.median(r) <= med_gate and r.max() <= 100 * med_gate, (precision, np.median(r), r.max())
        med, p999, mx = stats(a, ref)
        assert med <= med_gate and p999 <= 1e-3, (precision, med, p999)


def test_modelled_tails_match_row_kernels(env):
    torch, sc, shard = env
    w = ics.WORKLOADS["surrogate_n65536"]
    n = 1800
    d = ics.particle_load(n, 62, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    cfg = sc.Config(n_cut=w.n_cut, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, rho_bar=w.rho_bar, reorder_every=-1)

    def surrogate(sim):
        seeded_surrogate(sc, sim.ctx, 42, w.n_cut, w.n0)
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)

    def table(sim):
        sc.steps_cyl_build_tail_table(sim.ctx, 129, 17)
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)

    for setup in (surrogate, table):
        sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
        setup(sim)
        a = sim.forces()
        assert sc.steps_cyl_last_eval(sim.ctx)["symmetric"]
        sim.close()
        r = rel_err(a, row_forces(sc, shard, cfg, d, setup))
        assert np.median(r) <= 1e-6 and r.max() <= 1e-4, (setup.__name__, np.median(r), r.max())
    # the infinite window's table form against the oracle's infinite line
    cfg_inf = sc.Config(n_cut=0, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_TABLE,
                        background=sc.STEPS_BG_INFINITE, rho_bar=w.rho_bar, reorder_every=-1)
    sim = sc.Simulation(cfg_inf, d["pos"], d["vel"], d["m"], d["h"])
    a = sim.forces()
    assert sc.steps_cyl_last_eval(sim.ctx)["symmetric"]
    sim.close()
    idx = ics.subsample(n, 200, seed=3)
    ref = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx)
    ref += oracle.background_field(d["pos"][idx], ics.R_SIM, 0.0, 1.0, w.rho_bar, mode=2)
    med, _, mx = stats(a[idx], ref)
    assert med <= 1e-5 and mx <= 1e-3, (med, mx)


def test_straight_run_matches_row_kernels_and_oracle(env):
    # The production softening law (h_i + h_j <= 0.16 L) takes the straight-run
    # kernels of both modelled tails. Pairs inside their softening support exist
    # in this load, so the redo of softened steps runs as well. The row kernels
    # take the tiered calls throughout.
    torch, sc, shard = env
    w = ics.WORKLOADS["production_n65536"]
    n = 2600
    d = ics.particle_load(n, 65, w.M_tot, displaced=True, rho_bar=w.rho_bar, eps_law="ratio8")
    assert 2.0 * d["h"].max() < 0.5
    pos = d["pos"]
    dR = np.hypot(pos[:, None, 0] - pos[None, :, 0], pos[:, None, 1] - pos[None, :, 1])
    np.fill_diagonal(dR, np.inf)
    softened = np.nonzero((dR < d["h"][:, None] + d["h"][None, :]).any(1))[0]
    assert softened.size >= 20, softened.size
    cfg = sc.Config(n_cut=w.n_cut, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, rho_bar=w.rho_bar, reorder_every=-1)
    seeded = {}

    def surrogate(sim):
        seeded["net"] = seeded_surrogate(sc, sim.ctx, 44, w.n_cut, w.n0)
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)

    def table(sim):
        sc.steps_cyl_build_tail_table(sim.ctx, 129, 17)
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)

    for setup in (surrogate, table):
        sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
        setup(sim)
        a = sim.forces()
        ev = sc.steps_cyl_last_eval(sim.ctx)
        assert ev["symmetric"] and ev["straight_run"], ev
        sim.close()
        r = rel_err(a, row_forces(sc, shard, cfg, d, setup))
        assert np.median(r) <= 1e-6 and r.max() <= 1e-4, (setup.__name__, np.median(r), r.max())
        if setup is surrogate:
            w16, scfg = seeded["net"]
            idx = np.union1d(ics.subsample(n, 60, seed=5), softened[:40])
            ref = oracle.pair_field_surrogate(d["pos"], d["m"], d["h"], 1.0, 1.0, w16, scfg, idx=idx)
            ref += oracle.background_field(d["pos"][idx], ics.R_SIM, w.n_cut * 1.0, 1.0, w.rho_bar, mode=1)
            med, _, mx = stats(a[idx], ref)
            assert med <= 2e-6 and mx <= 1e-4, (med, mx)
    # the literal softening law of the learned-tail workloads keeps the tiered calls
    wl = ics.WORKLOADS["surrogate_n65536"]
    dl = ics.particle_load(n, 66, wl.M_tot, displaced=True, rho_bar=wl.rho_bar)
    assert 2.0 * dl["h"].max() >= 0.5
    sim = sc.Simulation(cfg, dl["pos"], dl["vel"], dl["m"], dl["h"])
    surrogate(sim)
    sim.forces()
    ev = sc.steps_cyl_last_eval(sim.ctx)
    assert ev["symmetric"] and not ev["straight_run"], ev
    sim.close()


def test_newton_third_law(env):
    # each pair enters both particles with opposite sign, so the net pair force
    # is left only with the rounding of the FP32 partial sums (the i side and
    # the j side of a pair are summed in different groups): far below the
    # 1e-6 that FP32 forces of every ordered pair reach
    torch, sc, shard = env
    d = ics.particle_load(3000, 63, 1.0)
    sim = sc.Simulation(sc.Config(n_cut=16, background=sc.STEPS_BG_OFF), d["pos"], d["vel"], d["m"], d["h"])
    a = sim.forces()
    sim.close()
    net = (d["m"][:, None] * a).sum(0)
    scale = (d["m"][:, None] * np.abs(a)).sum()
    assert np.all(np.abs(net) < 2e-8 * scale), net / scale


def test_tiny_softening_falls_back_to_row_kernels(env):
    torch, sc, shard = env
    d = ics.particle_load(700, 64, 1.0)
    d["h"] = d["h"].copy()
    d["h"][5] = 1e-9        # (L / h_min)^2 ~ 1e18: the fixed-point unit would be too coarse
    sim = sc.Simulation(sc.Config(n_cut=8), d["pos"], d["vel"], d["m"], d["h"])
    a = sim.forces()
    assert not sc.steps_cyl_last_eval(sim.ctx)["symmetric"]
    sim.close()
    med, p999, _ = stats(a, oracle_accel(d["pos"], d["m"], d["h"], 8))
    assert med <= 1e-5 and p999 <= 1e-3
