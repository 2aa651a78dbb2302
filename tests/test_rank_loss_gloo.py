"""Rank loss detected on the host, with three gloo ranks as spawned processes
and no GPU.

- A rank that crashes between steps is named by the others' Heartbeat before
  their next step, within the heartbeat's timeout.
- A rank that leaves on purpose is named at once.
- All ranks stepping together pass every heartbeat and collective.
- Without a heartbeat, the second line holds: a collective whose peer died
  ends with an error under the process group's short timeout, not a hang.

The heartbeat's key-value store lives in the test process, so it outlives any
rank. The failure is always made on the host (a process exit)."""
import datetime
import json
import multiprocessing
import os
import socket
import time

import pytest

WORLD = 3
HB_TIMEOUT = 2.0
PG_TIMEOUT = 5.0


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _record(out_dir, rank, **kw):
    with open(os.path.join(out_dir, f"{rank}.json"), "w") as fh:
        json.dump(kw, fh)


def worker(mode, rank, world, pg_port, hb_port, out_dir):
    import torch
    import torch.distributed as dist
    from paper_2602_20787_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(pg_port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=PG_TIMEOUT))
    store = dist.TCPStore("127.0.0.1", hb_port, None, False, timeout=datetime.timedelta(seconds=30))
    hb = shard.Heartbeat(store, rank, world, timeout=HB_TIMEOUT, prefix=mode)
    t = torch.ones(4, dtype=torch.float64)
    for step in range(6):
        if mode == "crash" and rank == 2 and step == 2:
            os._exit(3)                      # a crash between steps: nothing in flight
        if mode == "collective" and rank == 1 and step == 1:
            os._exit(3)                      # dies before the collective, without a heartbeat
        t0 = time.monotonic()
        if mode != "collective":
            try:
                hb.beat(step)
            except shard.RankLost as e:
                _record(out_dir, rank, lost=e.ranks, step=e.step, elapsed=time.monotonic() - t0)
                os._exit(0)                  # leave without entering the step's collective
        try:
            dist.all_reduce(t)
        except RuntimeError as e:
            _record(out_dir, rank, collective_error=type(e).__name__, step=step, elapsed=time.monotonic() - t0)
            os._exit(0)
        if mode == "leave" and rank == 1 and step == 1:
            hb.leave(step)
            _record(out_dir, rank, left=step)
            os._exit(0)
    _record(out_dir, rank, done=True, total=float(t[0]))
    dist.destroy_process_group()


def run(mode, tmp_path):
    import torch.distributed as dist
    hb_store = dist.TCPStore("127.0.0.1", 0, None, True, timeout=datetime.timedelta(seconds=30),
                             wait_for_workers=False)
    ctx = multiprocessing.get_context("spawn")
    pg_port = free_port()
    procs = [ctx.Process(target=worker, args=(mode, r, WORLD, pg_port, hb_store.port, str(tmp_path)))
             for r in range(WORLD)]
    for p in procs:
        p.start()
    deadline = time.monotonic() + 120.0
    for p in procs:
        p.join(max(deadline - time.monotonic(), 0.1))
    hung = [p for p in procs if p.is_alive()]
    for p in hung:
        p.kill()
        p.join()
    assert not hung, f"{len(hung)} rank(s) did not finish"
    res = {}
    for r in range(WORLD):
        path = tmp_path / f"{r}.json"
        res[r] = json.loads(path.read_text()) if path.exists() else None
    return [p.exitcode for p in procs], res


@pytest.fixture(autouse=True)
def _torch():
    pytest.importorskip("torch")


def test_ranks_stepping_together_pass(tmp_path):
    codes, res = run("all", tmp_path)
    assert codes == [0, 0, 0]
    for r in range(WORLD):
        assert res[r]["done"] and res[r]["total"] == WORLD ** 6


def test_crashed_rank_is_named_before_the_next_step(tmp_path):
    codes, res = run("crash", tmp_path)
    assert codes == [0, 0, 3]
    for r in (0, 1):
        assert res[r]["lost"] == [2] and res[r]["step"] == 2
        assert res[r]["elapsed"] < HB_TIMEOUT + 1.0
    assert res[2] is None


def test_rank_that_leaves_is_named_at_once(tmp_path):
    codes, res = run("leave", tmp_path)
    assert codes == [0, 0, 0]
    assert res[1] == {"left": 1}
    for r in (0, 2):
        assert res[r]["lost"] == [1] and res[r]["step"] == 2
        assert res[r]["elapsed"] < HB_TIMEOUT      # named by the leave() key, not by the timeout


def test_collective_with_a_dead_peer_errors_instead_of_hanging(tmp_path):
    codes, res = run("collective", tmp_path)
    assert codes == [0, 3, 0]
    for r in (0, 2):
        assert res[r]["step"] == 1 and res[r]["collective_error"]
        assert res[r]["elapsed"] < PG_TIMEOUT + 5.0


class DictStore:
    """In-memory stand-in for a torch.distributed store (set/check/delete_key)."""

    def __init__(self):
        self.d = {}

    def set(self, k, v):
        self.d[k] = v

    def check(self, keys):
        return all(k in self.d for k in keys)

    def delete_key(self, k):
        return self.d.pop(k, None) is not None


def test_heartbeat_logic_single_process():
    from paper_2602_20787_gb300 import shard
    st = DictStore()
    hb = shard.Heartbeat(st, 0, 3, timeout=0.05)
    for r in (1, 2):                              # the peers have posted step 0
        st.set(f"heartbeat/step/0/{r}", b"1")
    hb.beat(0)
    st.set("heartbeat/step/1/1", b"1")            # rank 2 never posts step 1
    with pytest.raises(shard.RankLost) as e:
        hb.beat(1)
    assert e.value.ranks == [2] and e.value.step == 1
    st.set("heartbeat/step/1/2", b"1")
    hb.beat(1)
    assert "heartbeat/step/0/0" not in st.d       # the previous step's own key is dropped
    shard.Heartbeat(st, 2, 3, timeout=0.05).leave(1)
    t0 = time.monotonic()
    with pytest.raises(shard.RankLost) as e:
        hb.beat(2)
    assert e.value.ranks == [2] and e.value.step == 2   # the leaver is named before the timeout
    assert time.monotonic() - t0 < 0.05
    for bad in (dict(rank=3, world=3), dict(rank=0, world=0), dict(rank=0, world=2, timeout=0.0)):
        with pytest.raises(ValueError):
            shard.Heartbeat(st, **bad)
