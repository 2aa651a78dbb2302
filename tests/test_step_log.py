"""The per-step JSONL log of Simulation.run, on the host: the chunking of the
KDK steps and the records, with the library calls replaced by fakes (no GPU)."""
import json

import numpy as np
import pytest

from paper_2602_20787_gb300 import steps_cyl as sc


def fake_sim(timing=(2.0e9, 4.0)):
    sim = sc.Simulation.__new__(sc.Simulation)
    sim.calls = []
    state = {"t": 0.0}

    def step(dt, k):
        sim.calls.append((dt, k))
        state["t"] += dt * k

    sim.step = step
    sim.diagnostics = lambda: np.array([1.0, 2.0, 3.0, 0.5, 0.25, 0.7, state["t"], 1.0])
    sim.last_timing = lambda: timing
    return sim


def test_chunks_and_records(tmp_path):
    sim = fake_sim()
    path = tmp_path / "run.jsonl"
    sim.run(0.01, 7, log=str(path), every=3)
    assert sim.calls == [(0.01, 3), (0.01, 3), (0.01, 1)]
    recs = [json.loads(x) for x in path.read_text().splitlines()]
    assert [r["step"] for r in recs] == [3, 6, 7]
    assert recs[-1]["t"] == pytest.approx(0.07) and recs[0]["a"] == 0.7
    assert recs[0]["P"] == [1.0, 2.0, 3.0] and recs[0]["L_z"] == 0.5 and recs[0]["mass"] == 1.0
    assert recs[0]["pair_images_per_s"] == pytest.approx(2.0e9 / 4.0e-3)
    assert all(r["wall_ms_per_step"] >= 0.0 for r in recs)
    sim.run(0.01, 2, log=str(path))          # appends
    assert len(path.read_text().splitlines()) == 5


def test_without_log_is_one_call():
    sim = fake_sim()
    sim.run(0.02, 9)
    assert sim.calls == [(0.02, 9)]


def test_untimed_evaluation_and_bad_chunk(tmp_path):
    sim = fake_sim(timing=(0.0, 0.0))
    path = tmp_path / "run.jsonl"
    sim.run(0.01, 1, log=str(path))
    assert json.loads(path.read_text())["pair_images_per_s"] is None
    with pytest.raises(ValueError):
        sim.run(0.01, 1, log=str(path), every=0)
