"""The symmetric kernels in the index-checked build (STEPS_DEBUG_INDEX=1: every
computed index of their shared and global accesses checked against its buffer,
an index outside recorded and clamped, the record folded into the device error
word). Where compute-sanitizer cannot run, the index-checked library stands in
for it: every symmetric form (plain Kahan and plain sums, learned tail, correction
table with each read, the straight-run instances of both modelled tails on the
production softening law, nearest-image table, infinite window, the symmetric
sharded step of two emulated ranks) runs on ragged sizes, and each call must
return without STEPS_EDEVICE and give the release build's forces.

The checked library is built and loaded in a child process
(STEPS_CYL_INDEX_CHECKED=1), so that the release library of the other tests
stays the one loaded in this process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.conftest import ROOT

pytestmark = pytest.mark.gpu

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2602_20787_gb300 import ics, shard, steps_cyl as sc
from tests.gpu_helpers import seeded_surrogate
out = {}
w = ics.WORKLOADS["surrogate_n65536"]
for n in (2, 129, 1000, 2500):
    d = ics.particle_load(n, 100 + n, w.M_tot, displaced=True, rho_bar=w.rho_bar)
    forms = {}
    for prec in (sc.STEPS_FP32_KAHAN, sc.STEPS_FP32_PLAIN):
        sim = sc.Simulation(sc.Config(n_cut=16, precision=prec, reorder_every=-1), d["pos"], d["vel"], d["m"], d["h"])
        forms["plain%d" % prec] = sim.forces()
        assert sc.steps_cyl_last_eval(sim.ctx)["symmetric"] or n < 3
        sim.close()
    base = dict(n_cut=w.n_cut, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, rho_bar=w.rho_bar, reorder_every=-1)
    sim = sc.Simulation(sc.Config(**base), d["pos"], d["vel"], d["m"], d["h"])
    seeded_surrogate(sc, sim.ctx, 42, w.n_cut, w.n0)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    forms["surrogate"] = sim.forces()
    for name, read in (("cic", sc.STEPS_TABLE_READ_CIC), ("tsc", sc.STEPS_TABLE_READ_TSC)):
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_FULL)
        sc.steps_cyl_set_table_read(sim.ctx, read)
        sc.steps_cyl_build_tail_table(sim.ctx, 65, 9, err_median=1.0, err_p999=1.0, check_particles=64)
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
        forms["table_" + name] = sim.forces()
    sim.close()
    # the production softening law (every h_i + h_j < L / 2): the straight-run
    # instances of the learned tail and the residual tables
    dp = ics.particle_load(n, 200 + n, w.M_tot, displaced=True, rho_bar=w.rho_bar, eps_law="ratio8")
    sim = sc.Simulation(sc.Config(**base), dp["pos"], dp["vel"], dp["m"], dp["h"])
    seeded_surrogate(sc, sim.ctx, 42, w.n_cut, w.n0)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    forms["surrogate_straight"] = sim.forces()
    ev = sc.steps_cyl_last_eval(sim.ctx)
    assert ev["straight_run"] or (n < 3 and not ev["symmetric"]), ev
    for name, read in (("cic", sc.STEPS_TABLE_READ_CIC), ("tsc", sc.STEPS_TABLE_READ_TSC)):
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_FULL)
        sc.steps_cyl_set_table_read(sim.ctx, read)
        sc.steps_cyl_build_tail_table(sim.ctx, 65, 9, err_median=1.0, err_p999=1.0, check_particles=64)
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
        forms["table_straight_" + name] = sim.forces()
        ev = sc.steps_cyl_last_eval(sim.ctx)
        assert ev["straight_run"] or (n < 3 and not ev["symmetric"]), ev
    sim.close()
    near = dict(base, n0=0)
    sim = sc.Simulation(sc.Config(**near), d["pos"], d["vel"], d["m"], d["h"])
    sc.steps_cyl_build_tail_table(sim.ctx, 65, 9, err_median=1.0, err_p999=1.0, check_particles=64)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    forms["nearest"] = sim.forces()
    sim.close()
    inf = dict(base, n_cut=0, tail=sc.STEPS_TAIL_TABLE, background=sc.STEPS_BG_INFINITE)
    sim = sc.Simulation(sc.Config(**inf), d["pos"], d["vel"], d["m"], d["h"])
    forms["infinite"] = sim.forces()
    sim.close()
    # the symmetric sharded step, two ranks emulated in turn on one GPU
    if n >= 1000:
        import torch
        sims = [sc.Simulation(sc.Config(n_cut=16, reorder_every=-1), d["pos"], d["vel"], d["m"], d["h"])
                for _ in range(2)]
        ranks = [shard.GpuRows(s, r, 2, symmetric=True) for r, s in enumerate(sims)]
        for _ in range(2):
            recv = torch.cat([r.drift(1e-4) for r in ranks], 0)       # the all-gather, in rank order
            tot = torch.stack([r.force(recv) for r in ranks], 0).sum(0)  # the reduce-scatter's sums
            k = tot.shape[0] // 2
            for q, r in enumerate(ranks):
                r.finish(tot[q * k:(q + 1) * k].contiguous())
        forms["sharded_state"] = sum(r.state() for r in ranks)
        for s in sims:
            s.close()
    out[str(n)] = {k: np.asarray(v, dtype=float).tolist() for k, v in forms.items()}
out["lib"] = sc.load()._name
print("RESULT " + json.dumps(out))
'''


def run_child(checked):
    env = dict(os.environ)
    env["STEPS_CYL_INDEX_CHECKED"] = "1" if checked else "0"
    code = "ROOT = %r\n" % ROOT + CHILD
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_index_checked_build_matches_release():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    checked = run_child(True)    # raises on STEPS_EDEVICE (an index outside its buffer)
    release = run_child(False)
    assert os.path.basename(checked.pop("lib")) == "libsteps_cyl_checked.so"
    assert os.path.basename(release.pop("lib")) == "libsteps_cyl.so"
    assert checked.keys() == release.keys()
    for n in checked:
        assert checked[n].keys() == release[n].keys()
        for form in checked[n]:
            a, b = np.array(checked[n][form]), np.array(release[n][form])
            assert np.all(np.isfinite(a)), (n, form)
            # the checks change no arithmetic: the same forces, bit for bit
            assert np.array_equal(a, b), (n, form, np.abs(a - b).max())
