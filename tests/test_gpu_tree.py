"""GPU tests of the octree (Sect. 2.4) against the FP64 oracle's tree: the same
frame gives the same interactions (counted exactly) and forces to FP32
precision; ragged sizes, leaf sizes and frames; the per-evaluation random
frames; the radial calibration and its correction; a KDK run with
checkpoint/resume; refused configurations and a particle outside the root."""
import math

import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics
from tests.gpu_helpers import stats, table_dR_max

pytestmark = pytest.mark.gpu

N0 = 4


@pytest.fixture(scope="module")
def sc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20787_gb300 import steps_cyl
    steps_cyl.load()
    return steps_cyl


def workload(n=3000, seed=3):
    w = ics.WORKLOADS["surrogate_n1048576"]
    return w, ics.particle_load(n, seed, w.M_tot, displaced=True, rho_bar=w.rho_bar)


def tree_config(sc, rho_bar, **kw):
    base = dict(n_cut=0, n0=N0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_TABLE,
                background=sc.STEPS_BG_INFINITE, rho_bar=rho_bar, force=sc.STEPS_FORCE_OCTREE, theta=0.5,
                leaf_size=16)
    base.update(kw)
    return sc.Config(**base)


def oracle_tree(d, rho_bar, zeta, phi, theta=0.5, leaf=16, idx=None):
    cfg = oracle.make_table_cfg(0, N0, 257, 33, table_dR_max(d["pos"]))
    g, st = oracle.tree_field(d["pos"], d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 0, theta, leaf, zeta, phi,
                              oracle.tail_table_build(cfg), cfg, idx=idx)
    sel = d["pos"] if idx is None else d["pos"][idx]
    return g + oracle.background_field(sel, ics.R_SIM, 0.0, 1.0, rho_bar, mode=2), st


def tree_sim(sc, w, d, zeta, phi, **kw):
    sim = sc.Simulation(tree_config(sc, w.rho_bar, **kw), d["pos"], d["vel"], d["m"], d["h"])
    sc.steps_cyl_tree_frame(sim.ctx, zeta, phi)
    return sim


@pytest.mark.parametrize("zeta,phi", [(0.37, 1.1), (0.0, 0.0), (0.999, -2.7)])
def test_tree_matches_oracle(sc, zeta, phi):
    w, d = workload()
    sim = tree_sim(sc, w, d, zeta, phi)
    a = sim.forces()
    st = sc.steps_cyl_tree_stats(sim.ctx)
    ref, ost = oracle_tree(d, w.rho_bar, zeta, phi)
    med, _, mx = stats(a, ref)
    print(f"frame ({zeta}, {phi}): median {med:.2e} max {mx:.2e}; nodes {st['nodes']} (oracle {ost[0]}), "
          f"interactions {st['interactions']:.0f} (oracle {ost[3]}), build {st['build_ms']:.2f} ms, "
          f"walk {st['walk_ms']:.2f} ms")
    assert st["nodes"] == ost[0] and st["depth"] == ost[2]
    assert st["interactions"] == ost[3]          # the same opening decisions, group by group
    assert med <= 1e-6 and mx <= 2e-5
    sim.close()


@pytest.mark.parametrize("n", [2, 31, 33, 129, 1000])
def test_tree_ragged_sizes(sc, n):
    w, d = workload(n, 50 + n)
    sim = tree_sim(sc, w, d, 0.2, 0.3, precision=sc.STEPS_FP32_PLAIN)
    ref, ost = oracle_tree(d, w.rho_bar, 0.2, 0.3)
    med, _, mx = stats(sim.forces(), ref)
    assert sc.steps_cyl_tree_stats(sim.ctx)["interactions"] == ost[3]
    assert med <= 2e-5 and mx <= 2e-3
    sim.close()


@pytest.mark.parametrize("leaf,theta", [(1, 0.5), (8, 0.3), (64, 0.8), (16, 1.0)])
def test_tree_leaf_sizes_and_angles(sc, leaf, theta):
    w, d = workload(2500, 9)
    sim = tree_sim(sc, w, d, 0.55, 0.9, leaf_size=leaf, theta=theta)
    ref, ost = oracle_tree(d, w.rho_bar, 0.55, 0.9, theta=theta, leaf=leaf)
    med, _, mx = stats(sim.forces(), ref)
    st = sc.steps_cyl_tree_stats(sim.ctx)
    assert st["nodes"] == ost[0] and st["interactions"] == ost[3]
    assert med <= 1e-6 and mx <= 2e-5
    sim.close()


def splitmix_frames(seed, first, count, L=1.0):
    # the library's per-evaluation frame draw (SplitMix64, state seed * golden + evaluation)
    M = (1 << 64) - 1
    out = []
    for e in range(first, first + count):
        s = (seed * 0x9E3779B97F4A7C15 + e) & M
        u = []
        for _ in range(2):
            s = (s + 0x9E3779B97F4A7C15) & M
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
            z ^= z >> 31
            u.append((z >> 11) * 2.0 ** -53)
        out.append((u[0] * L, 2.0 * math.pi * u[1]))
    return out


def test_random_frames_per_evaluation(sc):
    w, d = workload(2000, 11)
    sim = sc.Simulation(tree_config(sc, w.rho_bar, tree_seed=7), d["pos"], d["vel"], d["m"], d["h"])
    # init evaluated once (evaluation 0); the next two use draws 1 and 2
    frames = splitmix_frames(7, 1, 2)
    idx = ics.subsample(2000, 200, seed=4)
    for zeta, phi in frames:
        a = sim.forces()
        ref, _ = oracle_tree(d, w.rho_bar, zeta, phi, idx=idx)
        med, _, mx = stats(a[idx], ref)
        assert med <= 1e-6 and mx <= 2e-5
    assert sc.steps_cyl_tree_stats(sim.ctx)["evaluations"] == 3
    sim.close()


def test_radial_calibration_matches_oracle(sc):
    w, d = workload(2500, 13)
    sim = tree_sim(sc, w, d, 0.1, 0.2)
    frames = np.array([[0.13, 0.4], [0.71, 2.9], [0.42, -1.3]])
    sample = ics.subsample(2500, 600, seed=6)
    nb = 12
    tab, rmax = sc.steps_cyl_tree_calibrate(sim.ctx, 3, nb, 600, frames=frames, sample=sample)
    # the oracle's calibration: radial part of (tree - direct) in bins of rho
    cfg = oracle.make_table_cfg(0, N0, 257, 33, table_dR_max(d["pos"]))
    T = oracle.tail_table_build(cfg)
    direct = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, T, cfg, idx=sample)
    rho_all = np.hypot(d["pos"][:, 0], d["pos"][:, 1])
    assert rmax == pytest.approx(rho_all.max(), rel=1e-15)
    x, y = d["pos"][sample, 0], d["pos"][sample, 1]
    rho = np.hypot(x, y)
    k = np.minimum(nb - 1, (rho / rmax * nb).astype(int))
    sums, cnt = np.zeros(nb), np.zeros(nb)
    for zeta, phi in frames:
        g, _ = oracle.tree_field(d["pos"], d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 0, 0.5, 16, zeta, phi, T, cfg,
                                 idx=sample)
        e = ((g - direct)[:, 0] * x + (g - direct)[:, 1] * y) / rho
        np.add.at(sums, k, e)
        np.add.at(cnt, k, 1)
    ref = np.where(cnt > 0, sums / np.maximum(cnt, 1), 0.0)
    scale = np.median(np.linalg.norm(direct, axis=1))
    print("radial table", tab, "oracle", ref, "force scale", scale)
    assert np.abs(tab - ref).max() <= 1e-5 * scale
    # the corrected force subtracts the interpolated table along rho_hat
    a = sim.forces()
    ref_g, _ = oracle_tree(d, w.rho_bar, 0.1, 0.2)
    r = rho_all
    s_ = r / rmax * nb - 0.5
    kk = np.clip(np.floor(s_).astype(int), 0, nb - 2)
    t = np.clip(s_ - kk, 0.0, 1.0)
    D = np.where(s_ <= 0, tab[0], np.where(s_ >= nb - 1, tab[-1], (1 - t) * tab[kk] + t * tab[kk + 1]))
    ref_g[:, 0] -= D * d["pos"][:, 0] / r
    ref_g[:, 1] -= D * d["pos"][:, 1] / r
    med, _, mx = stats(a, ref_g)
    assert med <= 1e-6 and mx <= 1e-4    # relative to the corrected force, smaller near the axis
    # the same table installed in another context gives the same corrected forces
    other = tree_sim(sc, w, d, 0.1, 0.2)
    sc.steps_cyl_tree_set_radial(other.ctx, tab, rmax)
    np.testing.assert_array_equal(other.forces(), a)
    with pytest.raises(sc.StepsError):
        sc.steps_cyl_tree_set_radial(other.ctx, np.array([np.nan]), rmax)
    other.close()
    # removing it restores the plain tree force
    sc.steps_cyl_tree_calibrate(sim.ctx, 0)
    med, _, _ = stats(sim.forces(), oracle_tree(d, w.rho_bar, 0.1, 0.2)[0])
    assert med <= 1e-6
    sim.close()


def oracle_kdk_tree(d, rho_bar, frames, dt):
    # static space: kick dt/2, drift dt, kick dt/2, a new frame per force evaluation
    x, v = d["pos"].copy(), d["vel"].copy()
    dd = dict(d)

    def field(x, fr):
        dd["pos"] = x
        return oracle_tree(dd, rho_bar, *fr)[0]

    g = field(x, frames[0])
    for s in range(len(frames) - 1):
        v += 0.5 * dt * g
        x += dt * v
        x[:, 2] -= np.floor(x[:, 2])
        g = field(x, frames[s + 1])
        v += 0.5 * dt * g
    return x, v


def test_tree_kdk_and_resume(sc, tmp_path):
    w, d = workload(400, 17)
    d["vel"] = np.random.default_rng(3).normal(0.0, 0.02, d["pos"].shape)
    dt = 0.05
    frames = splitmix_frames(5, 0, 5)
    xo, vo = oracle_kdk_tree(d, w.rho_bar, frames, dt)
    sim = sc.Simulation(tree_config(sc, w.rho_bar, tree_seed=5), d["pos"], d["vel"], d["m"], d["h"])
    sim.step(dt, 2)
    path = str(tmp_path / "tree.ckpt")
    sim.checkpoint(path)
    sim.close()
    sim = sc.Simulation.resume(path)
    sim.step(dt, 2)
    xg, vg, _, t = sim.state()
    assert t == pytest.approx(4 * dt, rel=1e-14)
    assert sc.steps_cyl_tree_stats(sim.ctx)["evaluations"] == 5
    dx = xg - xo
    dx[:, 2] -= np.round(dx[:, 2])
    moved = np.abs(xo - d["pos"])
    moved[:, 2] = np.minimum(moved[:, 2], 1.0 - moved[:, 2])
    print(f"tree KDK: max position difference {np.abs(dx).max():.2e} of max displacement {moved.max():.2e}")
    assert np.abs(dx).max() <= 2e-4 * moved.max()
    assert np.abs(vg - vo).max() <= 2e-4 * np.abs(vo - d["vel"]).max()
    sim.close()


def test_tree_configurations_are_checked(sc):
    w, d = workload(300, 19)
    for kw in (dict(n_cut=16, tail=sc.STEPS_TAIL_TABLE), dict(theta=0.0), dict(theta=1.5), dict(leaf_size=0),
               dict(leaf_size=65), dict(precision=sc.STEPS_FP64), dict(force=2)):
        with pytest.raises(sc.StepsError) as e:
            sc.Simulation(tree_config(sc, w.rho_bar, **kw), d["pos"], d["vel"], d["m"], d["h"])
        assert e.value.code == sc.STEPS_EINVAL, kw
    sim = sc.Simulation(tree_config(sc, w.rho_bar), d["pos"], d["vel"], d["m"], d["h"])
    for call in (lambda: sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE),
                 lambda: sc.steps_cyl_tree_frame(sim.ctx, 1.0, 0.0)):
        with pytest.raises(sc.StepsError) as e:
            call()
        assert e.value.code in (sc.STEPS_EINVAL, sc.STEPS_ENOSURROGATE)
    sim.close()
    direct = sc.Simulation(sc.Config(), d["pos"], d["vel"], d["m"], d["h"])
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_tree_stats(direct.ctx)
    assert e.value.code == sc.STEPS_EINVAL
    direct.close()
    # a particle beyond the root cube is reported, not used
    pos = d["pos"].copy()
    pos[5, :2] = [0.9, 0.0]
    with pytest.raises(sc.StepsError) as e:
        sc.Simulation(tree_config(sc, w.rho_bar, R_sim=0.2), pos, d["vel"], d["m"], d["h"])
    assert e.value.code == sc.STEPS_EDEVICE


def test_tree_full_size_sampled(sc):
    # the benchmarked octree configuration: the production-shaped load (N = 524,288,
    # softening ratio 1:8), sampled particles against the oracle's walk of their groups
    w = ics.WORKLOADS["production_n524288"]
    d = ics.workload_ics(w)
    sim = sc.Simulation(tree_config(sc, w.rho_bar), d["pos"], d["vel"], d["m"], d["h"])
    sc.steps_cyl_tree_frame(sim.ctx, 0.4321, 2.2)
    a = sim.forces()
    st = sc.steps_cyl_tree_stats(sim.ctx)
    idx = ics.subsample(w.n, 64, seed=31)
    ref, ost = oracle_tree(d, w.rho_bar, 0.4321, 2.2, idx=idx)
    med, _, mx = stats(a[idx], ref)
    print(f"N = {w.n} octree: median {med:.2e} max {mx:.2e}; nodes {st['nodes']} (oracle {ost[0]}); "
          f"{st['interactions'] / w.n:.0f} interactions per particle; build {st['build_ms']:.1f} ms, "
          f"walk {st['walk_ms']:.1f} ms")
    assert st["nodes"] == ost[0] and st["depth"] == ost[2]
    # this load's net forces are small residuals: its FP32 forms sit near 2e-6 at the median
    assert med <= 1e-5 and mx <= 1e-3
    sim.close()


# ---- the R^3 octree ------------------------------------------------------------

def r3_tree_config(sc, rho_bar, **kw):
    base = dict(topology=sc.STEPS_TOPO_R3, n_cut=1, precision=sc.STEPS_FP32_KAHAN, background=sc.STEPS_BG_SPHERE,
                rho_bar=rho_bar, R_sim=2.0, force=sc.STEPS_FORCE_OCTREE, theta=0.5, leaf_size=16)
    base.update(kw)
    return sc.Config(**base)


def unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def oracle_tree_r3(d, cen, axis, angle, theta=0.5, leaf=16, idx=None):
    g, st = oracle.tree_field_r3(d["pos"], d["m"], d["h"], 1.0, 2.0, theta, leaf, cen, axis, angle, idx=idx)
    sel = d["pos"] if idx is None else d["pos"][idx]
    return g + oracle.background_sphere(sel, 1.0, d["rho_bar"]), st


@pytest.mark.parametrize("theta,leaf", [(0.5, 16), (0.3, 8), (0.8, 32)])
def test_r3_tree_matches_oracle(sc, theta, leaf):
    d = ics.ball_load(3000, 31)
    cen, axis, angle = [0.2, -0.3, 0.1], unit([0.3, -0.5, 0.8]), 1.3
    sim = sc.Simulation(r3_tree_config(sc, d["rho_bar"], theta=theta, leaf_size=leaf), d["pos"], d["vel"], d["m"],
                        d["h"])
    sc.steps_cyl_tree_frame_r3(sim.ctx, cen, axis, angle)
    a = sim.forces()
    st = sc.steps_cyl_tree_stats(sim.ctx)
    ref, ost = oracle_tree_r3(d, cen, axis, angle, theta, leaf)
    med, _, mx = stats(a, ref)
    print(f"R3 octree theta {theta}: median {med:.2e} max {mx:.2e}; nodes {st['nodes']} (oracle {ost[0]}), "
          f"interactions {st['interactions']:.0f} (oracle {ost[3]})")
    assert st["nodes"] == ost[0] and st["depth"] == ost[2] and st["interactions"] == ost[3]
    assert med <= 1e-6 and mx <= 2e-5
    sim.close()


def splitmix_frames_r3(seed, first, count, R_sim):
    # the library's R^3 frame draw: axis uniform on the sphere, angle, centre uniform in the ball of radius R_sim / 2
    M = (1 << 64) - 1
    out = []
    for e in range(first, first + count):
        s = (seed * 0x9E3779B97F4A7C15 + e) & M
        u = []
        for _ in range(6):
            s = (s + 0x9E3779B97F4A7C15) & M
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
            z ^= z >> 31
            u.append((z >> 11) * 2.0 ** -53)
        za, pa = 2.0 * u[0] - 1.0, 2.0 * math.pi * u[1]
        sa = math.sqrt(max(0.0, 1.0 - za * za))
        axis = [sa * math.cos(pa), sa * math.sin(pa), za]
        angle = 2.0 * math.pi * u[2]
        rc = 0.5 * R_sim * math.cbrt(u[3])
        zc, pc = 2.0 * u[4] - 1.0, 2.0 * math.pi * u[5]
        sc_ = math.sqrt(max(0.0, 1.0 - zc * zc))
        out.append(([rc * sc_ * math.cos(pc), rc * sc_ * math.sin(pc), rc * zc], axis, angle))
    return out


def test_r3_random_frames_per_evaluation(sc):
    d = ics.ball_load(2000, 32)
    sim = sc.Simulation(r3_tree_config(sc, d["rho_bar"], tree_seed=9), d["pos"], d["vel"], d["m"], d["h"])
    idx = ics.subsample(2000, 200, seed=4)
    for cen, axis, angle in splitmix_frames_r3(9, 1, 2, 2.0):
        a = sim.forces()
        ref, _ = oracle_tree_r3(d, cen, axis, angle, idx=idx)
        med, _, mx = stats(a[idx], ref)
        assert med <= 1e-6 and mx <= 2e-5
    sim.close()


def test_r3_radial_calibration_matches_oracle(sc):
    d = ics.ball_load(2500, 33)
    sim = sc.Simulation(r3_tree_config(sc, d["rho_bar"]), d["pos"], d["vel"], d["m"], d["h"])
    frames = [([0.1, 0.2, -0.3], unit([1, 1, 0.5]), 0.7), ([-0.4, 0.1, 0.2], unit([0.2, -1, 0.3]), 2.5)]
    flat = np.array([list(c) + list(a) + [g] for c, a, g in frames])
    sample = ics.subsample(2500, 500, seed=7)
    nb = 10
    tab, rmax = sc.steps_cyl_tree_calibrate(sim.ctx, 2, nb, 500, frames=flat, sample=sample)
    direct = oracle.pair_field_r3(d["pos"], d["m"], d["h"], 1.0, idx=sample)
    r = np.linalg.norm(d["pos"][sample], axis=1)
    assert rmax == pytest.approx(np.linalg.norm(d["pos"], axis=1).max(), rel=1e-15)
    k = np.minimum(nb - 1, (r / rmax * nb).astype(int))
    sums, cnt = np.zeros(nb), np.zeros(nb)
    for cen, axis, angle in frames:
        g, _ = oracle.tree_field_r3(d["pos"], d["m"], d["h"], 1.0, 2.0, 0.5, 16, cen, axis, angle, idx=sample)
        e = ((g - direct) * d["pos"][sample]).sum(1) / r
        np.add.at(sums, k, e)
        np.add.at(cnt, k, 1)
    ref = np.where(cnt > 0, sums / np.maximum(cnt, 1), 0.0)
    scale = np.median(np.linalg.norm(direct, axis=1))
    print("R3 radial table", tab, "oracle", ref)
    assert np.abs(tab - ref).max() <= 1e-5 * scale
    sim.close()


def test_r3_tree_configurations_are_checked(sc):
    d = ics.ball_load(300, 34)
    with pytest.raises(sc.StepsError) as e:
        sc.Simulation(r3_tree_config(sc, d["rho_bar"], precision=sc.STEPS_FP64), d["pos"], d["vel"], d["m"], d["h"])
    assert e.value.code == sc.STEPS_EINVAL
    sim = sc.Simulation(r3_tree_config(sc, d["rho_bar"]), d["pos"], d["vel"], d["m"], d["h"])
    for call in (lambda: sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE),
                 lambda: sc.steps_cyl_tree_frame(sim.ctx, 0.1, 0.2),
                 lambda: sc.steps_cyl_tree_frame_r3(sim.ctx, [0.0, 0.0, 0.0], [1.0, 1.0, 0.0], 0.3),
                 lambda: sc.steps_cyl_tree_frame_r3(sim.ctx, [2.0, 0.0, 0.0], [1.0, 0.0, 0.0], 0.3),
                 lambda: sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP64)):
        with pytest.raises(sc.StepsError) as e:
            call()
        assert e.value.code in (sc.STEPS_EINVAL, sc.STEPS_ENOSURROGATE)
    sim.close()


def test_r3_tree_kdk_resume_keeps_the_frame_sequence(sc, tmp_path):
    # random R^3 frames drawn by evaluation count, so a resumed run continues the sequence
    d = ics.ball_load(600, 35)
    d["vel"] = np.random.default_rng(5).normal(0.0, 0.01, d["pos"].shape)
    cfg = r3_tree_config(sc, d["rho_bar"], tree_seed=3)
    ref = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    ref.step(0.02, 4)
    xr, vr, _, _ = ref.state()
    ref.close()
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    sim.step(0.02, 2)
    path = str(tmp_path / "r3tree.ckpt")
    sim.checkpoint(path)
    sim.close()
    sim = sc.Simulation.resume(path)
    sim.step(0.02, 2)
    x, v, _, _ = sim.state()
    np.testing.assert_array_equal(x, xr)
    np.testing.assert_array_equal(v, vr)
    assert sc.steps_cyl_tree_stats(sim.ctx)["evaluations"] == 5
    sim.close()
