"""Pins of the oracle's octree (Sect. 2.4): with a vanishing opening angle the
tree walk is the direct sum of the same pair form; its error falls with the
opening angle; the key order is a Morton order of the frame; the field turns
with the load; the frame's shift along the axis changes only the tree."""
import math

import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics


def load(n, seed=3):
    w = ics.WORKLOADS["surrogate_n1048576"]
    return ics.particle_load(n, seed, w.M_tot, displaced=True, rho_bar=w.rho_bar)


def inf_table(pos, n0=4):
    dR_max = max(2.2 * float(np.hypot(pos[:, 0], pos[:, 1]).max()), 1.0)
    cfg = oracle.make_table_cfg(0, n0, 257, 33, dR_max)
    return oracle.tail_table_build(cfg), cfg


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.mark.parametrize("leaf", [1, 16])
def test_vanishing_angle_is_the_direct_sum(orc, leaf):
    d = load(700)
    tab, cfg = inf_table(d["pos"])
    g, st = oracle.tree_field(d["pos"], d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 0, 1e-7, leaf, 0.37, 1.1, tab, cfg)
    ref = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, tab, cfg)
    assert np.abs(g - ref).max() <= 1e-13 * np.abs(ref).max()
    assert st[3] == 700 * 700                       # every member against every particle, no node accepted
    # the plain window as the pair form
    g2, _ = oracle.tree_field(d["pos"], d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 8, 1e-7, leaf, 0.9, -2.0)
    ref2 = oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, 8)
    assert np.abs(g2 - ref2).max() <= 1e-13 * np.abs(ref2).max()


def test_error_falls_with_the_opening_angle(orc):
    d = load(3000)
    tab, cfg = inf_table(d["pos"])
    idx = ics.subsample(3000, 400, seed=1)
    ref = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, tab, cfg, idx=idx)
    med, inter = [], []
    for th in (0.15, 0.3, 0.5):
        g, st = oracle.tree_field(d["pos"], d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 0, th, 16, 0.21, 0.4, tab, cfg)
        med.append(np.median(rel(g[idx], ref)))
        inter.append(st[3])
    print("median errors", med, "interactions", inter)
    assert med[0] < 1e-4 and med[2] < 1e-2
    assert med[0] < med[1] < med[2]
    assert inter[0] > inter[1] > inter[2]
    # the sampled walk gives the same values for the listed particles
    gs, _ = oracle.tree_field(d["pos"], d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 0, 0.5, 16, 0.21, 0.4, tab, cfg,
                              idx=idx)
    np.testing.assert_array_equal(gs, g[idx])


def test_key_order_is_a_morton_order_of_the_frame(orc):
    d = load(2000)
    L, zeta, phi = 1.0, 0.61, 2.3
    key, order = oracle.tree_order(d["pos"], L, ics.R_SIM, zeta, phi)
    assert sorted(order.tolist()) == list(range(2000))
    assert np.all(np.diff(key.astype(np.float64)) >= 0)
    # the top three levels of each key against the particle's cell in the frame (FP64)
    S = 2.0 * max(L, 2.0 * ics.R_SIM)
    x, y, z = d["pos"][order].T
    c, s = math.cos(phi), math.sin(phi)
    zr = np.where(z + zeta >= L, z + zeta - L, z + zeta)
    u = np.stack([(c * x - s * y) / S + 0.5, (s * x + c * y) / S + 0.5, (zr - L / 2) / S + 0.5], 1)
    cell = np.floor(u * 8).astype(np.int64)
    top = (key >> np.uint64(54)).astype(np.int64)
    expect = np.zeros(2000, dtype=np.int64)
    for b in range(3):
        for a, sh in ((0, 2), (1, 1), (2, 0)):
            expect |= ((cell[:, a] >> b) & 1) << (3 * b + sh)
    near_edge = np.any(np.abs(u * 8 - np.round(u * 8)) < 1e-6, axis=1)
    assert np.all((top == expect) | near_edge)


def test_field_turns_with_the_load(orc):
    d = load(1500)
    tab, cfg = inf_table(d["pos"])
    a = 0.83
    Rz = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])
    g, _ = oracle.tree_field(d["pos"], d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 0, 0.5, 16, 0.3, 1.0, tab, cfg)
    # the turned load in the frame turned back by the same angle: the same tree
    g2, _ = oracle.tree_field(d["pos"] @ Rz.T, d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 0, 0.5, 16, 0.3, 1.0 - a, tab,
                              cfg)
    r = rel(g2, g @ Rz.T)
    assert np.median(r) < 1e-9
    assert np.mean(r < 1e-6) > 0.98      # group decisions taken on rounded inputs may flip at a boundary


def test_shift_along_the_axis_changes_only_the_tree(orc):
    # a different frame gives a different tree, whose error against the direct
    # sum stays of the same size; the mean radial error over frames is small
    d = load(2000)
    tab, cfg = inf_table(d["pos"])
    idx = ics.subsample(2000, 300, seed=2)
    ref = oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, tab, cfg, idx=idx)
    meds = []
    for zeta, phi in ((0.0, 0.0), (0.5, 0.0), (0.25, 2.0)):
        g, _ = oracle.tree_field(d["pos"], d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 0, 0.4, 16, zeta, phi, tab, cfg,
                                 idx=idx)
        meds.append(np.median(rel(g, ref)))
    print("per-frame median errors", meds)
    assert max(meds) < 3 * min(meds) and max(meds) < 1e-2


def test_particle_outside_the_root_is_refused(orc):
    d = load(200)
    pos = d["pos"].copy()
    pos[7, 0] = 2.0 * max(1.0, 2.0 * ics.R_SIM)       # beyond half the root side
    with pytest.raises(ValueError):
        oracle.tree_field(pos, d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 8, 0.5, 16, 0.0, 0.0)


# ---- the R^3 octree (Sect. 2.4: domain centre shifted inside R_sim / 2, rotation about a random axis) ----

def unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def test_r3_vanishing_angle_is_the_direct_sum(orc):
    d = ics.ball_load(800, 11)
    g, st = oracle.tree_field_r3(d["pos"], d["m"], d["h"], 1.0, 2.0, 1e-7, 8, [0.2, -0.3, 0.1], unit([1, 2, -1]), 0.9)
    ref = oracle.pair_field_r3(d["pos"], d["m"], d["h"], 1.0)
    assert np.abs(g - ref).max() <= 1e-13 * np.abs(ref).max()
    assert st[3] == 800 * 800


def test_r3_error_falls_with_the_opening_angle(orc):
    d = ics.ball_load(3000, 12)
    ref = oracle.pair_field_r3(d["pos"], d["m"], d["h"], 1.0)
    med = []
    for th in (0.2, 0.4, 0.7):
        g, _ = oracle.tree_field_r3(d["pos"], d["m"], d["h"], 1.0, 2.0, th, 16, [0.1, 0.4, -0.2], unit([0.3, -0.5, 0.8]),
                                    1.3)
        med.append(np.median(rel(g, ref)))
    print("R3 median errors", med)
    assert med[0] < 2e-4 and med[0] < med[1] < med[2] < 3e-2


def test_r3_field_turns_with_the_load(orc):
    # the load turned by Q, with the domain centre turned by Q and the frame rotation composed with Q^T,
    # sees the same tree: its field is the turned field
    d = ics.ball_load(1500, 13)
    ax, ang, cen = unit([0.3, -0.5, 0.8]), 1.3, np.array([0.1, 0.4, -0.2])
    g, _ = oracle.tree_field_r3(d["pos"], d["m"], d["h"], 1.0, 2.0, 0.5, 16, cen, ax, ang)
    # a quarter turn about the frame's own axis commutes with the frame rotation
    Q = rotation(ax, 0.5 * math.pi)
    g2, _ = oracle.tree_field_r3(d["pos"] @ Q.T, d["m"], d["h"], 1.0, 2.0, 0.5, 16, Q @ cen, ax, ang - 0.5 * math.pi)
    r = rel(g2, g @ Q.T)
    assert np.median(r) < 1e-9
    assert np.mean(r < 1e-6) > 0.98


def rotation(ax, ang):
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)
