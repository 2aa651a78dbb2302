"""Writes tests/golden/oracle_regression.json: the FP64 oracle's outputs on
small fixed inputs, one entry per oracle function.

The file is a regression record, not a pin. The pins that tie the oracle to the
paper and to the mathematics live in tests/test_oracle_*.py. This record makes
any later change to the oracle's arithmetic show up as a failing test and as a
diff of this file. Regenerate it only when such a change is intended, and name
in the commit message the passage of arXiv 2602.20787, or the reading of it,
that justifies the change.

It calls only oracle/ and the seeded input generator.

    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2602_20787_gb300 import ics  # noqa: E402

OUT = os.path.join(HERE, "oracle_regression.json")


def cases():
    """name -> (citation, zero-argument callable returning an array)."""
    d7 = ics.particle_load(7, 3, 1.0)
    ball = ics.ball_load(48, 2)
    ball400 = ics.ball_load(400, 2)  # large enough that the tree accepts nodes at theta = 0.5
    tree = lambda: oracle.tree_field_r3(ball400["pos"], ball400["m"], ball400["h"], 1.0, 2.0, 0.5, 4,
                                        [0.1, 0.2, -0.1], [0.0, 0.6, 0.8], 0.7)
    pts = np.array([[0.3, -0.1, 0.2], [1.7, 0.4, 0.9], [3.0, 2.0, 0.5], [-5.0, 0.5, 0.1], [0.0, 0.0, 0.0]])
    rh = [(0.0, 0.1), (0.03, 0.1), (0.05, 0.1), (0.07, 0.1), (0.1, 0.1), (0.4, 0.1)]
    smp = [(0.2, 0.1, 0.01), (1.5, -0.3, 0.2), (3.0, 0.5, 0.05), (0.01, 0.0, 0.3)]
    cosmo = oracle.make_cosmo()
    tcfg = oracle.make_table_cfg(16, 4, 9, 5, 6.0)
    w = ics.random_surrogate_params(5, 6.0)[:1250]
    u = np.array([[-0.5, 0.2, 0.9], [0.0, 0.0, 0.0], [1.0, -1.0, -0.3]])
    return {
        "spline_F": ("Eq. Force_spline_kernel",
                     lambda: np.array([oracle.spline_F(r, h) for r, h in rh])),
        "spline_F_over_r": ("Eq. Force_spline_kernel over r",
                            lambda: np.array([oracle.spline_F_over_r(r, h) for r, h in rh])),
        "image_force": ("Eq. ForceCylindrical",
                        lambda: np.array([oracle.image_force(p, 0.05, 1.0, 5)[0] for p in pts[:4]])),
        "pair_field": ("Eq. ComovingEquationsOfMotionCylindrical, pair term",
                       lambda: oracle.pair_field(d7["pos"], d7["m"], d7["h"], 1.0, 1.0, 3)),
        "cylinder_field": ("Eq. F_horiz (finite height)",
                           lambda: np.array([oracle.cylinder_field(r, 3.0, 8.0, 1.0, 0.7) for r in (0.1, 1.2, 2.9, 4.5)])),
        "background_field_finite": ("Eq. F_horiz",
                                    lambda: oracle.background_field(pts, 3.0, 8.0, 1.0, 0.7, mode=1)),
        "background_field_infinite": ("Eq. F_horiz_infty",
                                      lambda: oracle.background_field(pts, 3.0, 8.0, 1.0, 0.7, mode=2)),
        "hubble": ("Sect. 2.3 Friedmann equation",
                   lambda: np.array([oracle.hubble(cosmo, a) for a in (0.02, 0.1, 0.5, 1.0)])),
        "a_step": ("Sect. 2.3 Friedmann equation, one step",
                   lambda: np.array([oracle.a_step(cosmo, a, 0.01) for a in (0.02, 0.1, 0.5, 1.0)])),
        "tail_sums": ("Eq. ForceCylindrical, images |k| > n0",
                      lambda: np.array([oracle.tail_sums(a, b, c, 1.0, 16, 4) for a, b, c in smp])),
        "image_sums_inf": ("Sect. 2.2, Ncut -> infinity",
                           lambda: np.array([oracle.image_sums_inf(a, b, c, 4) for a, b, c in smp])),
        "tail_table_build": ("Sect. 2.3, eq. S1R2EwaldCorrectionTable",
                             lambda: oracle.tail_table_build(tcfg)),
        "mlp_forward": ("Learned tail network (3-32-32-2 ReLU)",
                        lambda: np.asarray(oracle.mlp_forward(w, u))),
        "pair_field_r3": ("Sect. 2.1, eq. NewtonianForce",
                          lambda: oracle.pair_field_r3(ball["pos"], ball["m"], ball["h"], 1.0)),
        "tree_field_r3": ("Sect. 2.4, octree", lambda: tree()[0]),
        "tree_field_r3_stats": ("Sect. 2.4, octree: node and interaction counts", lambda: tree()[1]),
    }


def main():
    oracle.build()
    rec = {}
    for name, (cite, fn) in cases().items():
        v = np.asarray(fn(), dtype=np.float64)
        rec[name] = {"cite": cite, "shape": list(v.shape), "values": [float(x) for x in v.ravel()]}
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")
    print(f"wrote {OUT} ({len(rec)} entries)")


if __name__ == "__main__":
    main()
