"""Shared helpers of the GPU parity tests: the oracle's total acceleration and
the per-particle relative error metric (median and 99.9th percentile of
|a - a_ref| / |a_ref|, the metric of the paper's force-accuracy figure)."""
import numpy as np

import oracle
from paper_2602_20787_gb300 import ics


def oracle_accel(pos, m, h, n_cut, idx=None, G=1.0, L=1.0, R=ics.R_SIM, rho0=None, background=1, a=1.0):
    if rho0 is None:
        rho0 = m.sum() / (np.pi * R * R * L)
    g = oracle.pair_field(pos, m, h, G, L, n_cut, idx=idx)
    sel = pos if idx is None else pos[idx]
    g += oracle.background_field(sel, R, n_cut * L, G, rho0, mode=background)
    return g / a ** 3


def rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


def stats(a, ref):
    r = rel_err(a, ref)
    return float(np.median(r)), float(np.quantile(r, 0.999)), float(r.max())


def seeded_surrogate(sc, ctx, seed, n_cut, n0, dR_max=8.0, mu=(0.02, -0.01), scale=(0.05, 0.03)):
    """Install a seeded network (weights from the input generator, not from the
    library's training) in a context with bounds that accept it, and return the
    oracle's view of it: the FP16-rounded weights the kernel uses and the
    surrogate configuration."""
    p = ics.random_surrogate_params(seed, dR_max, mu=mu, sc=scale)
    sc.steps_cyl_set_surrogate(ctx, p, err_median=1.0, err_p999=1.0)
    cfg = oracle.make_surr_cfg(n_cut, n0, float(p[1254]), (float(p[1250]), float(p[1251])),
                               (float(p[1252]), float(p[1253])))
    return p[:1250].astype(np.float16).astype(np.float64), cfg


def table_dR_max(pos, L=1.0):
    """The input range a table or network built with dR_max = 0 takes: 2.2 x the
    largest particle radius in units of L, at least 1."""
    return max(2.2 * float(np.hypot(pos[:, 0], pos[:, 1]).max()) / L, 1.0)
