"""The allocation-free entry point steps_cyl_pair_accel_noalloc, for callers
that may not allocate device memory (their device memory is budgeted by another
allocator, or they may not take cudaMalloc's device-wide synchronisation, or
they may allocate only while initialising). It is called through the C ABI and
checked against the FP64 oracle's pair field (static space, no background), on
calls in a row with different inputs, so a call cannot lean on what the
previous call left in the shared scratch array. One call fills the array to its
limit, STEPS_NOALLOC_MAX_N particles, so the last packed particle and the last
partial-sum slot are written and read. Outputs start as NaN, so a value the
call did not write shows.

This file is collected last so that a run stopping at the first failure has run
every other test before it."""
import numpy as np
import pytest

import oracle
from paper_2602_20787_gb300 import ics

pytestmark = pytest.mark.gpu

# the gate of the FP32 forms against the FP64 oracle (median, every sampled particle)
MEDIAN_TOL, MAX_TOL = 1e-5, 1e-3


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20787_gb300 import steps_cyl
    steps_cyl.load()
    return torch, steps_cyl


def noalloc_accel(torch, sc, d, n_cut, precision):
    dev = torch.device("cuda", torch.cuda.current_device())
    cols = [torch.tensor(np.ascontiguousarray(d["pos"][:, k]), device=dev) for k in range(3)]
    m = torch.tensor(d["m"], device=dev)
    h = torch.tensor(d["h"], device=dev)
    out = [torch.full_like(m, float("nan")) for _ in range(3)]
    stream = torch.cuda.current_stream(dev)
    sc.steps_cyl_pair_accel_noalloc(*cols, m, h, 1.0, 1.0, n_cut, precision, *out, stream=stream.cuda_stream)
    stream.synchronize()
    return torch.stack(out, 1).cpu().numpy()


def sample(n, k, seed):
    """k sampled particles plus the first and the last 64 (the ragged last block)."""
    idx = np.concatenate([np.arange(min(64, n)), np.arange(max(0, n - 64), n), ics.subsample(n, k, seed=seed)])
    return np.unique(idx)


def test_noalloc_matches_oracle_on_calls_in_a_row(env):
    torch, sc = env
    nmax = sc.STEPS_NOALLOC_MAX_N
    cases = [(ics.particle_load(5000, 41, 1.0), 16, sc.STEPS_FP32_KAHAN, 400),
             (ics.particle_load(nmax, 43, 1.0), 2, sc.STEPS_FP32_KAHAN, 256),
             (ics.particle_load(3001, 42, 1.0), 7, sc.STEPS_FP32_PLAIN, 400)]
    for d, n_cut, precision, k in cases:
        n = d["pos"].shape[0]
        got = noalloc_accel(torch, sc, d, n_cut, precision)
        assert np.all(np.isfinite(got)), "an output kept its NaN fill or is not finite"
        idx = sample(n, k, seed=n)
        ref = oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, n_cut, idx=idx)
        rel = np.linalg.norm(got[idx] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert np.median(rel) <= MEDIAN_TOL and rel.max() <= MAX_TOL, (n, np.median(rel), rel.max())


def test_noalloc_refuses_bad_arguments_without_launching(env):
    torch, sc = env
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 256
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    short = torch.zeros(n - 1, dtype=torch.float64, device=dev)
    host = np.zeros(n)
    # the binding: sizes beyond the limit, host arrays, unequal lengths
    big = torch.zeros(sc.STEPS_NOALLOC_MAX_N + 1, dtype=torch.float64, device=dev)
    for args in [(big,) * 5 + (big,) * 3, (host,) * 5 + (x,) * 3, (x,) * 5 + (x, x, short)]:
        with pytest.raises(sc.StepsError) as e:
            sc.steps_cyl_pair_accel_noalloc(*args[:5], 1.0, 1.0, 4, sc.STEPS_FP32_KAHAN, *args[5:])
        assert e.value.code == sc.STEPS_EINVAL
    # the C entry point itself: a size beyond the limit, and a host pointer among device pointers
    L = sc.load()
    p = sc._ptr(x)
    pb = sc._ptr(big)
    assert L.steps_cyl_pair_accel_noalloc(sc.STEPS_NOALLOC_MAX_N + 1, pb, pb, pb, pb, pb, 1.0, 1.0, 4,
                                          sc.STEPS_FP32_KAHAN, pb, pb, pb, None) == sc.STEPS_EINVAL
    ph = host.ctypes.data_as(sc.ctypes.c_void_p)
    assert L.steps_cyl_pair_accel_noalloc(n, p, p, p, p, p, 1.0, 1.0, 4, sc.STEPS_FP32_KAHAN, p, p, ph,
                                          None) == sc.STEPS_EINVAL
    torch.cuda.synchronize(dev)
