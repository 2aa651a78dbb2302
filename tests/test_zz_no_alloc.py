"""The allocation-free entry point steps_cyl_pair_accel_noalloc, for callers
that may not allocate device memory (their device memory is budgeted by another
allocator, or they may not take cudaMalloc's device-wide synchronisation, or
they may allocate only while initialising). It is checked through the C ABI
against the context entry point steps_cyl_forces (background off, static
space: the same pair term), on two calls in a row with different inputs, so a
call cannot lean on what the previous call left in the shared scratch array.

This file is collected last so that a run stopping at the first failure has run
every other test before it."""
import numpy as np
import pytest

from paper_2602_20787_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_20787_gb300 import steps_cyl
    steps_cyl.load()
    return torch, steps_cyl


def reference_accel(sc, d, n_cut, precision):
    # the context keeps the caller's particle order here, as the entry point does
    cfg = sc.Config(n_cut=n_cut, precision=precision, background=sc.STEPS_BG_OFF, reorder_every=-1)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    a = sim.forces()
    sim.close()
    return a


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


def test_noalloc_matches_context_path_on_two_calls(env):
    torch, sc = env
    cases = [(ics.particle_load(5000, 41, 1.0), 16, sc.STEPS_FP32_KAHAN),
             (ics.particle_load(3001, 42, 1.0), 7, sc.STEPS_FP32_PLAIN)]
    for d, n_cut, precision in cases:
        got = noalloc_accel(torch, sc, d, n_cut, precision)
        ref = reference_accel(sc, d, n_cut, precision)
        assert np.all(np.isfinite(got))
        # same kernels; the work split may differ, so agreement is to FP32
        # rounding, within the FP32 tolerance of the parity tests
        rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert np.median(rel) <= 1e-6 and rel.max() <= 1e-5, (np.median(rel), rel.max())


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    torch, sc = env
    n = sc.STEPS_NOALLOC_MAX_N + 1
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_pair_accel_noalloc(x, x, x, x, x, 1.0, 1.0, 4, sc.STEPS_FP32_KAHAN, x, x, x)
    assert e.value.code == sc.STEPS_EINVAL
    # the C entry point rejects it too, without launching anything
    L = sc.load()
    p = sc._ptr(x)
    assert L.steps_cyl_pair_accel_noalloc(n, p, p, p, p, p, 1.0, 1.0, 4, sc.STEPS_FP32_KAHAN, p, p, p, None) \
        == sc.STEPS_EINVAL
