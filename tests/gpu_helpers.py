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
