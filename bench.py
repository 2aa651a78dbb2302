"""Benchmark of the S1xR2 StePS hot path on GB300.

One step = one comoving KDK step (kick, drift + z wrap + repack, pair-force
kernel over every pair, background, kick) of the production-shaped workload:
N = 524,288 particles, Ncut = 64 (128 images per pair), softening ratio 1:8,
LCDM from a = 0.02, positions and momenta in FP64. The headline form is the
learned far-image tail: the near images |k| <= 4 summed exactly in FP32 with
Kahan-compensated sums, the tail beyond them from the network (trained on the
GPU first, accepted only within its error bound, re-checked against the plain
sum every 50 steps). The metric is equivalent pair-images per second: N (N-1)
128 per step, the work of the plain window sum the form stands in for, over
the whole job. The same line carries the plain FP32-Kahan 128-image sum timed
on the same run, both forms' errors against FP64, and the speedup.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       python bench.py --workload NAME   (the other workloads, one JSON line each)
Under torchrun (N > 1) the ranks share one cylinder (strong scaling): each owns
a contiguous range of rows, and each step all-gathers the packed rows once.

--impl reference times the FP64 CPU oracle (the deliberately plain reference of
this project) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "production_n524288"
CHECK_EVERY = 50     # the plain sum re-checks the learned tail every 50 KDK steps
REORDER_EVERY = 32   # the library's default Morton re-order interval
METRIC = "pair-interactions/s (images counted)"
UNIT = "pair-images/s"
MUFU_RSQRT_PER_SM_CLK = 16  # MUFU rsqrt lanes per SM per clock, measured on GB300 (one rsqrt per pair-image)


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


PROFILED = {  # the committed ncu summary of each timed kernel, and the sources that define it
    "plain": ("pair_sym_kahan_production_n524288.md", ["pair_fp32.cuh", "pair_sym.cuh"]),
    "surrogate": ("pair_sym_surr_kahan_production_n524288.md", ["pair_fp32.cuh", "surrogate_pair.cuh", "pair_sym.cuh"]),
}


def kernel_source_hash(kind: str = "plain") -> str:
    """A pair kernel's sources and its launch shape (the stream-K CTA multiplier)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_20787_gb300", "csrc")
    for f in PROFILED[kind][1]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "steps_cyl.cu")) as fh:
        h.update("".join(ln for ln in fh if ln.startswith("#define STEPS_CTA_MULT")).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kind: str = "plain"):
    """DRAM bytes per pair-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", PROFILED[kind][0])
    if not os.path.exists(path):
        return None
    src_hash, traffic = None, None
    with open(path) as fh:
        for ln in fh:
            if ln.startswith("kernel_source_sha256_16:"):
                src_hash = ln.split(":", 1)[1].strip()
            if ln.startswith("dram_bytes_per_launch:"):
                try:
                    traffic = float(ln.split(":", 1)[1].strip())
                except ValueError:
                    traffic = None
    if src_hash != kernel_source_hash(kind):
        return None
    return traffic


def cpu_baseline(w, d, target_s: float = 15.0):
    """FP64 oracle (as it stands) on a bounded i-sample of the same workload:
    pair field of the sampled i against all N particles plus the background.
    The sample is sized from a small probe and rescaled once from a real run,
    so that it takes about target_s seconds."""
    import oracle
    from paper_2602_20787_gb300 import ics
    n = w.n

    def run(k, seed):
        idx = ics.subsample(n, k, seed=seed)
        t0 = time.perf_counter()
        oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, w.n_cut, idx=idx)
        oracle.background_field(d["pos"][idx], ics.R_SIM, w.n_cut * 1.0, 1.0, w.rho_bar, mode=1)
        return time.perf_counter() - t0

    dt_probe = max(run(16, 777), 1e-3)
    k = int(min(n, max(16, 16 * target_s / dt_probe)))
    el = run(k, 778)
    if el < 0.5 * target_s and k < n:
        k = int(min(n, max(k + 1, k * target_s / max(el, 1e-3))))
        el = run(k, 779)
    images = k * (n - 1) * 2.0 * w.n_cut
    return {"value": images / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{k} i-particles x all {n} j x {2 * w.n_cut} images (FP64 pair field + background), {el:.1f} s"}


def oracle_rate(call, n_all, units_per_i, unit, what, target_s=4.0, seed=779):
    """The FP64 oracle (as it stands) timed beside a form on a bounded i-sample:
    call(idx) evaluates the sampled particles; one i stands for units_per_i
    work units (pairs, or 1 for a force per particle)."""
    import oracle
    from paper_2602_20787_gb300 import ics
    probe = ics.subsample(n_all, 4, seed=seed)
    t0 = time.perf_counter()
    call(probe)
    dt_probe = max(time.perf_counter() - t0, 1e-3)
    k = int(min(n_all, max(4, 4 * target_s / dt_probe)))
    for attempt in range(2):  # the probe carries start-up costs: rescale once from a real run
        idx = ics.subsample(n_all, k, seed=seed + 1)
        t0 = time.perf_counter()
        call(idx)
        el = time.perf_counter() - t0
        if attempt == 0 and el < 0.5 * target_s and k < n_all:
            k = int(min(n_all, max(k + 1, k * target_s / max(el, 1e-3))))
        else:
            break
    return {"value": k * units_per_i / el, "unit": unit, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{k} i-particles: {what}, {el:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2602_20787_gb300 import ics
    import oracle
    oracle.build()
    w = ics.WORKLOADS[WORKLOAD]
    d = ics.workload_ics(w)
    n = w.n
    per_step_target = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    # size the per-step sample from a real (untimed) calibration run, so that the
    # thread pool is warm and each step holds enough rows to keep every core busy
    k = 8 * oracle.num_threads()
    for _ in range(2):
        idx = ics.subsample(n, k, seed=900)
        t0 = time.perf_counter()
        oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, w.n_cut, idx=idx)
        el = max(time.perf_counter() - t0, 1e-3)
        k = int(min(n, max(8 * oracle.num_threads(), k * per_step_target / el)))
    times = []
    for s in range(args.warmup + args.steps):
        idx = ics.subsample(n, k, seed=1000 + s)
        t0 = time.perf_counter()
        oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, w.n_cut, idx=idx)
        oracle.background_field(d["pos"][idx], ics.R_SIM, w.n_cut * 1.0, 1.0, w.rho_bar, mode=1)
        el = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(el)
    images = k * (n - 1) * 2.0 * w.n_cut
    value = images * len(times) / sum(times)
    sample = f"each step: {k} i-particles x all {n} j x {2 * w.n_cut} images (FP64 oracle pair field + background)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (FP64 oracle, plain window sum)", "n": n, "n_cut": w.n_cut,
                   "i_sample_per_step": k},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measured_peaks():
    """The measured copy-bandwidth and bf16 GEMM peaks of the GB300 (MEASURED_PEAKS.json), or None."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


def surrogate_roofline(n_sm, sm_mhz, n0, pairs, kernel_s, symmetric=False, headline=True):
    """Roofline of the learned-tail pair kernel per pair (one i, one j):
    - MUFU: 2 n0 + 1 near-image rsqrt, 4 rsqrt + 2 rcp of the two-sided
      continuum base and 1 rsqrt of dR, at 16 MUFU ops/SM/clk;
    - tensor: the network's own 2 (3 x 32 + 32 x 32 + 32 x 2) = 2368 flops at
      the measured sustained dense f16/bf16 rate (the kernel runs inside a
      seconds-long step).
    The larger time per pair binds. pairs: the pairs the kernel evaluated (each
    unordered pair once for the symmetric kernels). headline: the committed ncu
    DRAM figure belongs to the headline launch; other workloads report None."""
    mufu_ops = (2 * n0 + 1) + 4 + 2 + 1
    mlp_flops = 2 * (3 * 32 + 32 * 32 + 32 * 2)
    pk = measured_peaks()
    if pk and pk.get("bf16_tflops_sustained"):
        tensor_flops, tensor_src = pk["bf16_tflops_sustained"] * 1e12, "of measured (bf16 sustained, same rate as f16)"
    else:
        tensor_flops, tensor_src = 1.7e15, "of fallback (sustained bf16)"
    mufu_pairs = n_sm * sm_mhz * 1e6 * MUFU_RSQRT_PER_SM_CLK / mufu_ops
    tensor_pairs = tensor_flops / mlp_flops
    peak = min(mufu_pairs, tensor_pairs)
    achieved = pairs / kernel_s
    return {"bound": "alu" if mufu_pairs <= tensor_pairs else "tensor", "achieved": achieved, "peak": peak,
            "unit": "pair interactions evaluated/s", "frac": achieved / peak,
            "traffic": recorded_traffic("surrogate") if headline else None, "symmetric": symmetric,
            "peak_basis": f"min(MUFU: {n_sm} SMs x {MUFU_RSQRT_PER_SM_CLK}/SM/clk x {sm_mhz:.0f} MHz / {mufu_ops} "
                          f"ops per pair = {mufu_pairs:.3e}; tensor: {tensor_flops:.3e} flop/s {tensor_src} / "
                          f"{mlp_flops} network flops per pair = {tensor_pairs:.3e})"}


def force_errors(sim, sc, idx, forms):
    """Relative force errors of the FP32 forms against the library's FP64 form
    (which the test-suite pins to the FP64 oracle at <= 1.4e-13) on the sampled
    particles, all at the same state. forms: {name: tail}."""
    out = {}
    for name, tail in forms.items():
        sc.steps_cyl_set_tail(sim.ctx, tail)
        out[name] = sim.forces_subset(idx)
    sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP64)
    a64 = sim.forces_subset(idx)
    sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP32_KAHAN)
    return {k: _err(v, a64) for k, v in out.items()}


def run_sharded(args, rank, world, local):
    """N > 1 GPUs: one cylinder of the headline workload strong-scaled across
    the ranks. Every rank builds the same context from the same load, trains
    the same network (deterministic), and then owns a contiguous range of rows
    (steps_cyl_shard); each KDK step is drift, one NCCL all-gather of the packed
    rows, the rank's share of the unordered pairs, one reduce-scatter of the
    integer pair sums, and the finish of its rows (shard.ShardedSimulation).
    value = the whole cylinder's equivalent pair-images per second over the
    slowest rank's time."""
    import torch
    import torch.distributed as dist
    from paper_2602_20787_gb300 import ics, shard, steps_cyl as sc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)
    w = ics.WORKLOADS[WORKLOAD]
    d = ics.workload_ics(w)
    n = w.n
    t0, dt = ics.run_schedule(w)
    cfg = sc.Config(n_cut=w.n_cut, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_FULL,
                    background=sc.STEPS_BG_FINITE, comoving=True, a_start=w.a_start, t_start=t0, rho_bar=w.rho_bar,
                    check_particles=1024, device=local, stream=stream.cuda_stream)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    try:
        sc.steps_cyl_train_surrogate(sim.ctx, sc.steps_cyl_train_cfg_default())
        accepted = True
    except sc.StepsError as e:
        if e.code != sc.STEPS_ESURROGATE_REJECTED:
            raise
        accepted = False
    tail = sc.STEPS_TAIL_SURROGATE if accepted else sc.STEPS_TAIL_FULL
    sc.steps_cyl_set_tail(sim.ctx, tail)
    rows = shard.GpuRows(sim, rank, world)
    ssim = shard.ShardedSimulation(rows, tail=tail if accepted else 0, check_every=CHECK_EVERY)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    ssim.step(dt, args.warmup)
    dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    if rank == 0:
        clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    pair_ms = []
    for s in range(args.steps):
        flush.fill_(float(s))
        ev[s][0].record(stream)
        ssim.step(dt, 1)
        ev[s][1].record(stream)
        pair_ms.append(sc.steps_cyl_last_timing(sim.ctx)[1])
    torch.cuda.synchronize(dev)
    dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    t_local = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    t_max = shard.max_over_ranks(t_local, device=dev)
    kernel_max = shard.max_over_ranks(statistics.mean(pair_ms) / 1e3, device=dev)
    pairs = n * (n - 1.0)
    images_per_step = pairs * 2.0 * w.n_cut
    value = images_per_step * args.steps / t_max

    # end to end through the public API: per step the sharded KDK step and the
    # whole cylinder's diagnostics read back to the host (inputs stay resident;
    # the only per-step traffic is the device-side all-gather)
    te0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ssim.step(dt, 1)
        ssim.diagnostics()
    torch.cuda.synchronize(dev)
    te = shard.max_over_ranks(time.perf_counter() - te0, device=dev)
    diag = ssim.diagnostics()

    if rank == 0:
        props = torch.cuda.get_device_properties(dev)
        sm_mhz = clk["sm_max_mhz"] or 2070.0
        roof = surrogate_roofline(props.multi_processor_count, sm_mhz, w.n0, rows.chunk * (n - 1.0), kernel_max,
                                  headline=False)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD + (" (learned tail, n0 = 4)" if accepted else
                                               " (plain sum: network rejected)"),
                       "n": n, "n_cut": w.n_cut, "n0": w.n0, "parallelism": f"row shards x {world}",
                       "exchange": ("per step one NCCL all-gather of the packed rows (32 B per particle) and one "
                                    "reduce-scatter of the int64 pair sums (24 B per particle); each unordered pair "
                                    "evaluated once across the ranks") if rows.symmetric else
                                   "one NCCL all-gather of the packed rows (32 B per particle) per step",
                       "rows_per_rank": rows.chunk, "a_after": float(diag[6]),
                       "l2": "256 MiB buffer written between timed steps (inputs 16 MB < L2)"},
            "kdk_step_ms": 1e3 * t_max / args.steps,
            "pair_kernel_ms": 1e3 * kernel_max,
            "roofline": roof,
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
            "e2e": {"value": images_per_step * args.e2e_steps / te, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 8 * 8 * world, "steps": args.e2e_steps} if args.e2e_steps > 0 else None,
            "gpu_launches": 5 * args.steps * world,
            "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    dist.barrier()
    sim.close()
    dist.destroy_process_group()
    return 0


def run(args):
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        return run_sharded(args, rank, world, local)

    import torch
    from paper_2602_20787_gb300 import ics, steps_cyl as sc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = ics.WORKLOADS[WORKLOAD]
    d = ics.workload_ics(w)
    n = w.n
    t0, dt = ics.run_schedule(w)
    cfg = sc.Config(n_cut=w.n_cut, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_FULL,
                    background=sc.STEPS_BG_FINITE, comoving=True, a_start=w.a_start, t_start=t0, rho_bar=w.rho_bar,
                    check_every=CHECK_EVERY, check_particles=1024, device=local, stream=stream.cuda_stream)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    ctx = sim.ctx

    # the learned tail: trained by the library's own GPU kernels on its FP64 tail
    # sums, then accepted only if it meets the error bound against the plain sum
    tr0 = time.perf_counter()
    try:
        rep = sc.steps_cyl_train_surrogate(ctx, sc.steps_cyl_train_cfg_default())
        accepted = True
    except sc.StepsError as e:
        if e.code != sc.STEPS_ESURROGATE_REJECTED:
            raise
        rep, accepted = e.report, False
    train_wall_s = time.perf_counter() - tr0
    sc.steps_cyl_set_tail(ctx, sc.STEPS_TAIL_SURROGATE if accepted else sc.STEPS_TAIL_FULL)

    # L2 flush buffer (larger than the 129 MB L2), written between timed steps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed_steps(k):
        """k KDK steps, each bracketed by CUDA events on the context stream with
        an L2 flush between them; returns (per-step ms, pair-kernel ms)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        pair = []
        for s in range(k):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            sc.steps_cyl_kdk_step(ctx, dt, 1)  # synchronises to read the device error word
            ev[s][1].record(stream)
            pair.append(sc.steps_cyl_last_timing(ctx)[1])
        torch.cuda.synchronize(dev)
        return [a.elapsed_time(b) for a, b in ev], pair

    for _ in range(args.warmup):
        sc.steps_cyl_kdk_step(ctx, dt, 1)
    torch.cuda.synchronize(dev)
    steps_before = args.warmup
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    clocks.start()
    torch.cuda.synchronize(dev)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    step_ms, pair_ms = timed_steps(args.steps)
    g1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    region_ms = g0.elapsed_time(g1)
    t_steps = sum(step_ms) / 1e3
    pairs = n * (n - 1.0)
    images_per_step = pairs * 2.0 * w.n_cut   # the window's equivalent images
    value = images_per_step * args.steps / t_steps
    kernel_s = statistics.mean(pair_ms) / 1e3
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clk["sm_max_mhz"] or 2070.0
    ev_s = sc.steps_cyl_last_eval(ctx)  # the pairs the kernel evaluated (each unordered pair once if symmetric)
    roof = surrogate_roofline(props.multi_processor_count, sm_mhz, w.n0, ev_s["pairs_evaluated"], kernel_s,
                              ev_s["symmetric"])
    peak_plain = props.multi_processor_count * MUFU_RSQRT_PER_SM_CLK * sm_mhz * 1e6
    if not accepted:  # the plain sum ran: its own roofline
        done = ev_s["pairs_evaluated"] * 2.0 * w.n_cut
        roof = {"bound": "alu", "achieved": done / kernel_s, "peak": peak_plain, "unit": "pair-images evaluated/s",
                "frac": done / kernel_s / peak_plain, "traffic": recorded_traffic("plain"),
                "symmetric": ev_s["symmetric"]}
    # reorders and surrogate checks that fell in the timed region add launches
    timed = range(steps_before + 1, steps_before + args.steps + 1)
    reorders = sum(1 for s in timed if s % REORDER_EVERY == 0)
    checks = sum(1 for s in timed if s % CHECK_EVERY == 0) if accepted else 0
    launches = 3 * args.steps + 12 * reorders + 6 * checks
    steps_before += args.steps

    # the plain FP32-Kahan image sum on the same run, for the speedup
    plain_steps = max(2, args.steps // 5)
    sc.steps_cyl_set_tail(ctx, sc.STEPS_TAIL_FULL)
    sc.steps_cyl_kdk_step(ctx, dt, 1)
    plain_ms, plain_pair_ms = timed_steps(plain_steps)
    steps_before += 1 + plain_steps
    plain_kernel_s = statistics.mean(plain_pair_ms) / 1e3
    plain_step_s = statistics.mean(plain_ms) / 1e3
    ev_p = sc.steps_cyl_last_eval(ctx)
    plain_done = ev_p["pairs_evaluated"] * 2.0 * w.n_cut
    sc.steps_cyl_set_tail(ctx, sc.STEPS_TAIL_SURROGATE if accepted else sc.STEPS_TAIL_FULL)
    sc.steps_cyl_kdk_step(ctx, dt, 1)  # the switch marks the forces stale: refresh them untimed

    # end to end through the public API with pinned host buffers: per step the
    # state goes host -> device (set_state), one KDK step runs, the state comes back
    e2e = None
    if args.e2e_steps > 0:
        host = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(6)]
        sc.steps_cyl_get_state(ctx, *host)
        torch.cuda.synchronize(dev)
        te0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sc.steps_cyl_set_state(ctx, *host)
            sc.steps_cyl_kdk_step(ctx, dt, 1)
            sc.steps_cyl_get_state(ctx, *host)
        torch.cuda.synchronize(dev)
        te = time.perf_counter() - te0
        e2e = {"value": images_per_step * args.e2e_steps / te, "unit": UNIT, "h2d_bytes_per_step": 6 * 8 * n,
               "d2h_bytes_per_step": 6 * 8 * n, "steps": args.e2e_steps}

    # force errors of both forms against FP64 at the same state, on the seeded sample
    idx = ics.subsample(n, 4096, seed=12345)
    forms = {"surrogate": sc.STEPS_TAIL_SURROGATE, "plain": sc.STEPS_TAIL_FULL} if accepted else \
        {"plain": sc.STEPS_TAIL_FULL}
    errs = force_errors(sim, sc, idx, forms)
    diag = sim.diagnostics()
    sim.close()

    cpu = None if args.no_cpu_baseline else cpu_baseline(w, d)
    ms_step = 1e3 * t_steps / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + (" (learned tail, n0 = 4)" if accepted else " (plain sum: network rejected)"),
                   "n": n, "n_cut": w.n_cut, "n0": w.n0, "images_per_pair_equivalent": 2 * w.n_cut,
                   "executed_near_images_per_pair": 2 * w.n0 + 1 if accepted else 2 * w.n_cut,
                   "form": "learned far-image tail + FP32-Kahan near images" if accepted else "plain FP32-Kahan",
                   "precision": "fp32 pair math, Kahan j-sum, fp64 state", "softening": "1:8 ratio law",
                   "background": "finite cylinder", "cosmology": "LCDM 0.3/0.7", "a_after": diag[5],
                   "check_every": CHECK_EVERY,
                   "l2": "256 MiB buffer written between timed steps (inputs 16 MB < L2)",
                   "timed_region_ms": region_ms},
        "kdk_step_ms": ms_step,
        "pair_kernel_ms": 1e3 * kernel_s,
        "surrogate": {"accepted": accepted, "train_ms": float(rep[5]), "train_wall_s": train_wall_s,
                      "check_vs_plain_median": float(rep[2]), "check_vs_plain_p999": float(rep[3]),
                      "error_vs_fp64": errs.get("surrogate"),
                      "speedup_vs_plain_kdk_step": plain_step_s / (ms_step / 1e3),
                      "speedup_vs_plain_pair_kernel": plain_kernel_s / kernel_s},
        "plain": {"steps": plain_steps, "kdk_step_ms": 1e3 * plain_step_s, "pair_kernel_ms": 1e3 * plain_kernel_s,
                  "pair_images_per_s": images_per_step / plain_step_s,
                  "error_vs_fp64": errs["plain"],
                  "roofline": {"bound": "alu", "achieved": plain_done / plain_kernel_s, "peak": peak_plain,
                               "unit": "pair-images evaluated/s", "frac": plain_done / plain_kernel_s / peak_plain,
                               "traffic": recorded_traffic("plain"), "symmetric": ev_p["symmetric"],
                               "peak_basis": f"{props.multi_processor_count} SMs x {MUFU_RSQRT_PER_SM_CLK} MUFU "
                                             f"rsqrt/SM/clk x {sm_mhz:.0f} MHz; 1 rsqrt per pair-image"}},
        "error_reference": "library FP64 form on 4096 particles (seed 12345), pinned to the FP64 oracle in the tests",
        "roofline": roof,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
        "e2e": e2e,
        "gpu_launches": launches,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Other workloads (python bench.py --workload NAME): one JSON line each. The
# reference for force errors is this library's FP64 form on a particle sample
# (parity-tested against the FP64 oracle in the test-suite).
# ---------------------------------------------------------------------------
def _ctx_for(sc, torch, w, d, precision, **kw):
    from paper_2602_20787_gb300 import ics
    t0, _ = ics.run_schedule(w)
    cfg = sc.Config(n_cut=w.n_cut, n0=w.n0, precision=precision, rho_bar=w.rho_bar, comoving=w.comoving,
                    a_start=w.a_start if w.comoving else 1.0, t_start=t0 if w.comoving else 0.0,
                    stream=torch.cuda.current_stream().cuda_stream, **kw)
    return sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])


def _timed_forces(sc, torch, sim, reps):
    dev = torch.device("cuda")
    out = [torch.empty(sim.n, dtype=torch.float64, device=dev) for _ in range(3)]
    ms = []
    for _ in range(reps):
        sc.steps_cyl_forces(sim.ctx, *out)
        ms.append(sc.steps_cyl_last_timing(sim.ctx)[1])
    torch.cuda.synchronize()
    return torch.stack(out, 1).cpu().numpy(), statistics.median(ms)


def _err(a, ref):
    r = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    return {"median": float(np.median(r)), "p999": float(np.quantile(r, 0.999)), "max": float(r.max())}


def run_r3_or_glass(args):
    """R^3 topology (N = 65,536 ball) and glass making (repulsive comoving
    S1xR2 run, N = 65,536): force / KDK-step timing and their checks."""
    import torch
    from paper_2602_20787_gb300 import ics, steps_cyl as sc
    n = 65536
    props = torch.cuda.get_device_properties(0)
    peak = props.multi_processor_count * MUFU_RSQRT_PER_SM_CLK * 2070e6
    stream = torch.cuda.current_stream().cuda_stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.workload == "r3_n65536":
        d = ics.ball_load(n, 11)
        cfg = sc.Config(topology=sc.STEPS_TOPO_R3, n_cut=1, background=sc.STEPS_BG_SPHERE, rho_bar=d["rho_bar"],
                        R_sim=2.0, comoving=True, a_start=0.1, t_start=ics.lcdm_time_of_a(0.1), stream=stream)
        sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
        a32, ms = _timed_forces(sc, torch, sim, 3)
        idx = ics.subsample(n, 256, seed=12345)
        sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP64)
        a64 = sim.forces_subset(idx)
        sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP32_KAHAN)
        pairs = n * (n - 1.0)
        dt = 0.01 * ics.lcdm_time_of_a(0.1)
        ev0.record()
        sim.step(dt, 10)
        ev1.record()
        torch.cuda.synchronize()
        import oracle
        cpu = oracle_rate(lambda ix: oracle.pair_field_r3(d["pos"], d["m"], d["h"], 1.0, idx=ix), n, n - 1.0,
                          "pair interactions/s", f"FP64 R3 pair field, all {n} j")
        line = {"workload": args.workload, "n": n, "topology": "R3", "images_per_pair": 1, "cpu_baseline": cpu,
                "fp32_kahan": {"pair_ms": ms, "pair_interactions_per_s": pairs / (ms * 1e-3),
                               "fraction_of_mufu_bound": pairs / (ms * 1e-3) / peak,
                               "error_vs_fp64": _err(a32[idx], a64)},
                "kdk": {"steps": 10, "step_ms": ev0.elapsed_time(ev1) / 10}}
    else:
        w = ics.WORKLOADS["lcdm_n65536"]
        d = ics.particle_load(n, 21, w.M_tot, rho_bar=w.rho_bar)
        a0, t0 = 0.02, ics.lcdm_time_of_a(0.02)
        cfg = sc.Config(G=-1.0, n_cut=16, rho_bar=w.rho_bar, comoving=True, a_start=a0, t_start=t0, stream=stream)
        sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])

        def rms_field():
            _, _, a, _ = sim.state()
            g = sim.forces() * a ** 3
            return math.sqrt((g ** 2).sum(1).mean())

        r0, t, steps, ms_tot = rms_field(), t0, 0, 0.0
        for _ in range(5):
            ev0.record()
            sim.step(0.03 * t, 25)
            ev1.record()
            torch.cuda.synchronize()
            ms_tot += ev0.elapsed_time(ev1)
            steps += 25
            t = sim.state()[3]
        line = {"workload": args.workload, "n": n, "topology": "S1R2", "G": -1.0, "n_cut": 16,
                "kdk": {"steps": steps, "step_ms": ms_tot / steps, "a_end": sim.state()[2],
                        "pair_images_per_s": n * (n - 1.0) * 32 / (ms_tot / steps * 1e-3),
                        "rms_net_field_ratio": rms_field() / r0}}
    sim.close()
    print(json.dumps(line), flush=True)
    return 0


def run_inf(args):
    """Infinite window (Ncut -> infinity, n_cut = 0) on the N = 65,536 load of
    the learned-tail law: the correction table carries the whole image line
    beyond the 2 n0 + 1 near images, with the infinite-cylinder background.
    Force and KDK-step timing and the pipe roofline of the table kernel; its
    errors are checked against the FP64 oracle in the test-suite (an infinite
    window has no GPU FP64 form to compare with here)."""
    import torch
    from paper_2602_20787_gb300 import ics, steps_cyl as sc
    w = ics.WORKLOADS["surrogate_n65536"]
    d = ics.workload_ics(w)
    n = w.n
    pairs = n * (n - 1.0)
    props = torch.cuda.get_device_properties(0)
    t0, _ = ics.run_schedule(w)
    cfg = sc.Config(n_cut=0, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_TABLE,
                    background=sc.STEPS_BG_INFINITE, rho_bar=w.rho_bar, comoving=True, a_start=w.a_start,
                    t_start=t0, stream=torch.cuda.current_stream().cuda_stream)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    _, ms = _timed_forces(sc, torch, sim, 3)
    evl = sc.steps_cyl_last_eval(sim.ctx)
    mufu = (2 * w.n0 + 1) + 2 + 2 + 1   # near images, infinite base rsqrt/rcp, the dR rsqrt
    peak = props.multi_processor_count * 2070e6 * MUFU_RSQRT_PER_SM_CLK / mufu
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dt = 0.01 * t0
    ev0.record()
    sim.step(dt, 10)
    ev1.record()
    torch.cuda.synchronize()
    line = {"workload": "inf_n65536", "n": n, "n_cut": "infinite", "n0": w.n0, "background": "infinite cylinder",
            "table": {"pair_ms": ms, "pair_interactions_per_s": pairs / (ms * 1e-3),
                      "executed_near_images_per_pair": 2 * w.n0 + 1,
                      "roofline": {"bound": "mufu", "mufu_ops_per_pair": mufu, "peak_pairs_per_s": peak,
                                   "achieved_pairs_evaluated_per_s": evl["pairs_evaluated"] / (ms * 1e-3),
                                   "frac": evl["pairs_evaluated"] / (ms * 1e-3) / peak,
                                   "symmetric": evl["symmetric"]},
                      "kdk_step_ms": ev0.elapsed_time(ev1) / 10}}
    import oracle
    tab, dR_max = sc.steps_cyl_get_tail_table(sim.ctx)
    ocfg = oracle.make_table_cfg(0, w.n0, tab.shape[1], tab.shape[0],
                                 max(2.2 * float(np.hypot(d["pos"][:, 0], d["pos"][:, 1]).max()), 1.0))
    otab = oracle.tail_table_build(ocfg)
    line["cpu_baseline"] = oracle_rate(
        lambda ix: oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, otab, ocfg, idx=ix), n, n - 1.0,
        "pair interactions/s", f"FP64 infinite-window table form, all {n} j")
    # the learned tail trained to infinity, checked against the table form
    rep = sc.steps_cyl_train_surrogate(sim.ctx, sc.steps_cyl_train_cfg_default())
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
    _, mss = _timed_forces(sc, torch, sim, 3)
    line["surrogate"] = {"train_ms": rep[5], "check_vs_table_median": rep[2], "check_vs_table_p999": rep[3],
                         "pair_ms": mss, "pair_interactions_per_s": pairs / (mss * 1e-3),
                         "table_speedup_over_surrogate": mss / ms}
    # the same table built by the Ewald summation of the line (Sect. 2.3), on the
    # paper's 144 x 128 grid at its single-precision setting, against the direct one
    sc.steps_cyl_build_tail_table(sim.ctx, 144, 128, dR_max)
    sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
    a_dir, _ = _timed_forces(sc, torch, sim, 1)
    rep_e = sc.steps_cyl_build_tail_table_ewald(sim.ctx, 144, 128, dR_max, 1.0, 5, 12)
    a_ew, mse = _timed_forces(sc, torch, sim, 3)
    line["ewald_table"] = {"nx": 144, "ny": 128, "alpha": 1.0, "nmax": 5, "mmax": 12, "build_ms": rep_e[2],
                           "direct_build_ms": rep_e[3], "max_node_difference": rep_e[0], "max_node": rep_e[1],
                           "pair_ms": mse, "forces_vs_direct_table": _err(a_ew, a_dir)}
    sim.close()
    # the paper's table over the nearest image alone (n0 = 0) on its 144 x 128
    # grid, against the exact line on a small sample, beside the n0 = 4 table
    idx = ics.subsample(n, 48, seed=12345)
    bg = oracle.background_field(d["pos"][idx], ics.R_SIM, 0.0, 1.0, w.rho_bar, mode=2)
    exact = oracle.pair_field_inf(d["pos"], d["m"], d["h"], 1.0, 1.0, idx=idx) + bg
    cfg0 = sc.Config(n_cut=0, n0=0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_TABLE,
                     background=sc.STEPS_BG_INFINITE, rho_bar=w.rho_bar, comoving=True, a_start=w.a_start,
                     t_start=t0, stream=torch.cuda.current_stream().cuda_stream)
    sim0 = sc.Simulation(cfg0, d["pos"], d["vel"], d["m"], d["h"])
    paper = {}
    for name, read in (("cic", sc.STEPS_TABLE_READ_CIC), ("tsc", sc.STEPS_TABLE_READ_TSC)):
        sc.steps_cyl_set_table_read(sim0.ctx, read)
        sc.steps_cyl_build_tail_table_ewald(sim0.ctx, 144, 128)
        a0, ms0 = _timed_forces(sc, torch, sim0, 3)
        paper[name] = {"pair_ms": ms0, "error_vs_exact_line": _err(a0[idx] * w.a_start ** 3, exact)}
    sim0.close()
    line["paper_table_nearest_image"] = {"n0": 0, "nx": 144, "ny": 128, "construction": "Ewald", **paper,
                                         "sample": "48 i-particles (seed 12345), FP64 oracle's infinite line"}
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    sc.steps_cyl_build_tail_table_ewald(sim.ctx, 144, 128)
    a4, _ = _timed_forces(sc, torch, sim, 1)
    line["paper_table_nearest_image"]["n0_4_table_error_vs_exact_line"] = _err(a4[idx] * w.a_start ** 3, exact)
    sim.close()
    print(json.dumps(line), flush=True)
    return 0


def run_table1(args):
    """The paper's tessellated particle load (Sect. 3.1, Fig. 4) in Table 1's
    geometry in units of L_z (R_sim = 0.5, D_S = 0.07, omega_c = 1.63973; N =
    65,536: 4 equal-mass core rings and 12 outer rings of 64 x 64 cells),
    comoving at Table 1's initial redshift (a = 0.02) and cosmology, Ncut = 16:
    the FP32-Kahan force and KDK-step times, the pair kernel's MUFU roofline,
    the error against the GPU FP64 form on a sample, and the oracle beside it."""
    import torch
    from paper_2602_20787_gb300 import ics, steps_cyl as sc
    d = ics.table1_load()
    n, n_cut = d["pos"].shape[0], 16
    pairs = n * (n - 1.0)
    props = torch.cuda.get_device_properties(0)
    peak = props.multi_processor_count * MUFU_RSQRT_PER_SM_CLK * 2070e6
    a0 = ics.TABLE1_A_INIT
    t0 = ics.lcdm_time_of_a(a0, ics.TABLE1_OMEGA_M, ics.TABLE1_OMEGA_L)
    R = ics.TABLE1_GEOMETRY["R_sim"]
    cfg = sc.Config(n_cut=n_cut, precision=sc.STEPS_FP32_KAHAN, R_sim=R, rho_bar=d["rho_bar"], comoving=True,
                    Omega_m=ics.TABLE1_OMEGA_M, Omega_L=ics.TABLE1_OMEGA_L, a_start=a0, t_start=t0,
                    stream=torch.cuda.current_stream().cuda_stream)
    sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
    a32, ms = _timed_forces(sc, torch, sim, 3)
    evl = sc.steps_cyl_last_eval(sim.ctx)
    idx = ics.subsample(n, 256, seed=12345)
    sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP64)
    a64 = sim.forces_subset(idx)
    sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP32_KAHAN)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    sim.step(0.01 * t0, 10)
    ev1.record()
    torch.cuda.synchronize()
    rate = pairs * 2 * n_cut / (ms * 1e-3)
    done = evl["pairs_evaluated"] * 2 * n_cut / (ms * 1e-3)   # pair-images the kernel evaluated per second
    line = {"workload": "table1_n65536", "n": n, "n_cut": n_cut, "core_rings": d["rings"].n_in,
            "outer_rings": d["rings"].n_out, "cells_per_ring": [64, 64],
            "mass_range": float(d["m"].max() / d["m"].min()),
            "fp32_kahan": {"pair_ms": ms, "pair_images_per_s": rate, "roofline_frac": done / peak,
                           "symmetric": evl["symmetric"],
                           "kdk_step_ms": ev0.elapsed_time(ev1) / 10, "error_vs_fp64": _err(a32[idx], a64)}}
    sim.close()
    import oracle

    def ref(ix):
        return (oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, n_cut, idx=ix)
                + oracle.background_field(d["pos"][ix], R, n_cut * 1.0, 1.0, d["rho_bar"], mode=1))
    line["cpu_baseline"] = oracle_rate(ref, n, (n - 1.0) * 2 * n_cut, "pair-images/s",
                                       f"FP64 oracle pair field + background, all {n} j x {2 * n_cut} images")
    print(json.dumps(line), flush=True)
    return 0


def run_octree(args):
    """Octree (Sect. 2.4) on the production-shaped load (softening ratio 1:8;
    N = 524,288, or 65,536 with the same law), infinite window with the
    correction table, Theta = 0.5, leaves of 16: build and walk time,
    interactions, the walk's pipe roofline, the time of the direct sum of the
    same pair form, errors and the mean radial force ratio against it on a
    particle sample, with and without the radial correction, and a KDK step.
    (Under the literal softening law of the other workloads most pairs overlap
    in softening, no node can stand in for its particles, and the tree does the
    direct sum's work.)"""
    import torch
    from paper_2602_20787_gb300 import ics, steps_cyl as sc
    w = ics.WORKLOADS["production_n524288"]
    n = 524288 if args.workload == "octree_n524288" else 65536
    d = ics.workload_ics(w, n=n)
    props = torch.cuda.get_device_properties(0)
    stream = torch.cuda.current_stream().cuda_stream
    common = dict(n_cut=0, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_TABLE,
                  background=sc.STEPS_BG_INFINITE, rho_bar=w.rho_bar, stream=stream)
    sim = sc.Simulation(sc.Config(force=sc.STEPS_FORCE_OCTREE, theta=0.5, leaf_size=16, **common), d["pos"],
                        d["vel"], d["m"], d["h"])
    reps, runs = 3, []
    for _ in range(reps):
        _timed_forces(sc, torch, sim, 1)
        runs.append(sc.steps_cyl_tree_stats(sim.ctx))
    st = min(runs, key=lambda r: r["build_ms"] + r["walk_ms"])
    mufu = (2 * w.n0 + 1) + 2 + 2 + 1   # per interaction: near images, infinite base rsqrt/rcp, the dR rsqrt
    peak = props.multi_processor_count * 2070e6 * MUFU_RSQRT_PER_SM_CLK / mufu
    rate = st["interactions"] / (st["walk_ms"] * 1e-3)
    line = {"workload": args.workload, "n": n, "n_cut": "infinite", "n0": w.n0, "theta": 0.5, "leaf_size": 16,
            "octree": {"build_ms": st["build_ms"], "walk_ms": st["walk_ms"],
                       "force_ms": st["build_ms"] + st["walk_ms"], "nodes": st["nodes"], "depth": st["depth"],
                       "interactions_per_particle": st["interactions"] / n,
                       "roofline": {"bound": "mufu", "mufu_ops_per_interaction": mufu, "peak_per_s": peak,
                                    "achieved_per_s": rate, "frac": rate / peak}}}
    # accuracy against the direct sum of the same pair form (GPU, FP32-Kahan) on a sample
    idx = ics.subsample(n, 2048, seed=12345)
    direct = sc.Simulation(sc.Config(**common), d["pos"], d["vel"], d["m"], d["h"])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    ad = direct.forces_subset(idx)
    ev1.record()
    torch.cuda.synchronize()
    line["direct_force_ms"] = ev0.elapsed_time(ev1)
    direct.close()

    def errors(a):
        # relative error of the net force (pair + background; on this near-homogeneous load
        # the pair sum is ~15x the net force, so the tree's pair-sum error is magnified), and
        # the mean radial error over the mean force magnitude (the bias the correction removes)
        r = np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1)
        x, y = d["pos"][idx, 0], d["pos"][idx, 1]
        rho = np.hypot(x, y)
        e_rad = ((a - ad)[:, 0] * x + (a - ad)[:, 1] * y) / rho
        return {"median": float(np.median(r)), "p99": float(np.quantile(r, 0.99)),
                "mean_radial_error_over_mean_force": float(np.mean(e_rad) / np.mean(np.linalg.norm(ad, axis=1)))}

    line["octree"]["error_vs_direct"] = errors(sim.forces_subset(idx))
    ev0.record()
    sc.steps_cyl_tree_calibrate(sim.ctx, 8, 32, 8192)
    ev1.record()
    torch.cuda.synchronize()
    line["octree"]["calibration_ms"] = ev0.elapsed_time(ev1)
    line["octree"]["error_vs_direct_radially_corrected"] = errors(sim.forces_subset(idx))
    # a tighter opening angle on the same load
    tight = sc.Simulation(sc.Config(force=sc.STEPS_FORCE_OCTREE, theta=0.3, leaf_size=16, **common), d["pos"],
                          d["vel"], d["m"], d["h"])
    a3 = tight.forces_subset(idx)
    st3 = sc.steps_cyl_tree_stats(tight.ctx)
    line["octree_theta_0.3"] = {"force_ms": st3["build_ms"] + st3["walk_ms"],
                                "interactions_per_particle": st3["interactions"] / n, "error_vs_direct": errors(a3)}
    tight.close()
    line["octree"]["speedup_vs_direct"] = line["direct_force_ms"] / (st["build_ms"] + st["walk_ms"])
    t0, _ = ics.run_schedule(w)
    ev0.record()
    sim.step(0.01 * t0 if t0 > 0 else 1e-3, 5)
    ev1.record()
    torch.cuda.synchronize()
    line["octree"]["kdk_step_ms"] = ev0.elapsed_time(ev1) / 5
    sim.close()
    import oracle
    ocfg = oracle.make_table_cfg(0, w.n0, 257, 33, max(2.2 * float(np.hypot(d["pos"][:, 0], d["pos"][:, 1]).max()), 1.0))
    otab = oracle.tail_table_build(ocfg)
    line["octree"]["forces_per_s"] = n / ((st["build_ms"] + st["walk_ms"]) * 1e-3)
    line["octree"]["cpu_baseline"] = oracle_rate(
        lambda ix: oracle.tree_field(d["pos"], d["m"], d["h"], 1.0, 1.0, ics.R_SIM, 0, 0.5, 16, 0.3, 0.7, otab, ocfg,
                                     idx=ix), n, 1.0, "particle forces/s",
        f"FP64 octree (sort, build, group walks of the sampled particles) of all {n}")
    print(json.dumps(line), flush=True)
    return 0


def run_octree_r3(args):
    """The R^3 octree (Sect. 2.4) on a uniform ball of 2^20 particles
    (softenings 0.02 .. 0.2, Theta = 0.5, leaves of 16): build and walk time,
    interactions, against the direct R^3 kernel on the same load (time and
    errors on a sample), and the FP64 oracle's octree timed beside it."""
    import torch
    from paper_2602_20787_gb300 import ics, steps_cyl as sc
    n = 1 << 20
    d = ics.ball_load(n, 41)
    stream = torch.cuda.current_stream().cuda_stream
    # the pair force alone: in a uniform ball the radial background term cancels it down to Poisson noise,
    # which would turn any tree error into a large relative error of the net force
    common = dict(topology=sc.STEPS_TOPO_R3, n_cut=1, precision=sc.STEPS_FP32_KAHAN, background=sc.STEPS_BG_OFF,
                  rho_bar=d["rho_bar"], R_sim=2.0, stream=stream)
    sim = sc.Simulation(sc.Config(force=sc.STEPS_FORCE_OCTREE, theta=0.5, leaf_size=16, **common), d["pos"], d["vel"],
                        d["m"], d["h"])
    runs = []
    for _ in range(3):
        _timed_forces(sc, torch, sim, 1)
        runs.append(sc.steps_cyl_tree_stats(sim.ctx))
    st = min(runs, key=lambda r: r["build_ms"] + r["walk_ms"])
    idx = ics.subsample(n, 2048, seed=12345)
    at = sim.forces_subset(idx)
    sim.close()
    direct = sc.Simulation(sc.Config(**common), d["pos"], d["vel"], d["m"], d["h"])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    ad = direct.forces_subset(idx)
    ev1.record()
    torch.cuda.synchronize()
    direct.close()
    r = np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1)
    import oracle
    cpu = oracle_rate(lambda ix: oracle.tree_field_r3(d["pos"], d["m"], d["h"], 1.0, 2.0, 0.5, 16, [0.1, 0.2, -0.1],
                                                      [0.0, 0.6, 0.8], 1.0, idx=ix), n, 1.0, "particle forces/s",
                      f"FP64 R3 octree (sort, build, group walks of the sampled particles) of all {n}")
    force_ms = st["build_ms"] + st["walk_ms"]
    line = {"workload": "octree_r3_n1048576", "n": n, "theta": 0.5, "leaf_size": 16,
            "octree": {"build_ms": st["build_ms"], "walk_ms": st["walk_ms"], "force_ms": force_ms,
                       "nodes": st["nodes"], "depth": st["depth"], "interactions_per_particle": st["interactions"] / n,
                       "forces_per_s": n / (force_ms * 1e-3),
                       "pair_error_vs_direct": {"median": float(np.median(r)), "p99": float(np.quantile(r, 0.99))},
                       "cpu_baseline": cpu},
            "direct_force_ms": ev0.elapsed_time(ev1), "speedup_vs_direct": ev0.elapsed_time(ev1) / force_ms}
    print(json.dumps(line), flush=True)
    return 0


def run_octree_accuracy(args):
    """The octree's accuracy in the manner of the paper's Fig. 3, on an evolved
    snapshot: the production-shaped load (softening 1:8, N = 65,536) is run
    with the direct sum of the infinite window from a = 0.02 to a = 1 in 1000
    comoving KDK steps. At a = 0.1, 0.3 and 1 the octree force (Theta = 0.3 ..
    0.8, with and without the radial correction calibrated at the start) is
    compared with the direct force on a particle sample: median relative error
    and mean radial and tangential force ratios."""
    import torch
    from paper_2602_20787_gb300 import ics, steps_cyl as sc
    w = ics.WORKLOADS["production_n524288"]
    n = 65536
    d = ics.workload_ics(w, n=n)
    t0, _ = ics.run_schedule(w)
    t1 = ics.lcdm_time_of_a(1.0, w.Omega_m, w.Omega_L)
    common = dict(n_cut=0, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, tail=sc.STEPS_TAIL_TABLE,
                  background=sc.STEPS_BG_INFINITE, rho_bar=w.rho_bar, comoving=True, a_start=w.a_start, t_start=t0,
                  stream=torch.cuda.current_stream().cuda_stream)
    sim = sc.Simulation(sc.Config(**common), d["pos"], d["vel"], d["m"], d["h"])
    # radial tables from the initial load, one per opening angle
    thetas = (0.3, 0.5, 0.8)
    tables = {}
    for th in thetas:
        tr = sc.Simulation(sc.Config(force=sc.STEPS_FORCE_OCTREE, theta=th, **common), d["pos"], d["vel"], d["m"],
                           d["h"])
        tables[th] = sc.steps_cyl_tree_calibrate(tr.ctx, 8, 32, 8192)
        tr.close()
    idx = ics.subsample(n, 4096, seed=12345)
    steps, out, done, ev0, ev1 = 1000, {}, 0, torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dt = (t1 - t0) / steps
    ms = 0.0
    for a_target in (0.1, 0.3, 1.0):
        t_target = ics.lcdm_time_of_a(a_target, w.Omega_m, w.Omega_L)
        k = int(round((t_target - t0) / dt)) - done
        ev0.record()
        sim.step(dt, k)
        ev1.record()
        torch.cuda.synchronize()
        ms += ev0.elapsed_time(ev1)
        done += k
        x, v, a, t = sim.state()
        ad = sim.forces_subset(idx)
        rho = np.hypot(x[idx, 0], x[idx, 1])
        er = np.stack([x[idx, 0] / rho, x[idx, 1] / rho], 1)
        et = np.stack([-er[:, 1], er[:, 0]], 1)
        fr_d = (ad[:, :2] * er).sum(1)
        ft_d = (ad[:, :2] * et).sum(1)
        rows = {}
        for th in thetas:
            for corr in (False, True):
                cfg = sc.Config(force=sc.STEPS_FORCE_OCTREE, theta=th, **dict(common, a_start=a, t_start=t))
                tr = sc.Simulation(cfg, x, v, d["m"], d["h"])
                if corr:   # the table calibrated on the initial load, as the paper does
                    sc.steps_cyl_tree_set_radial(tr.ctx, *tables[th])
                at = tr.forces_subset(idx)
                tr.close()
                r = np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1)
                rows[f"theta_{th}" + ("_corrected" if corr else "")] = {
                    "median_rel_err": float(np.median(r)), "mean_rel_err": float(np.mean(r)),
                    "median_radial_ratio": float(np.median((at[:, :2] * er).sum(1) / fr_d)),
                    "median_tangential_ratio": float(np.median((at[:, :2] * et).sum(1) / ft_d)),
                    "mean_radial_error_over_mean_force": float(np.mean(((at - ad)[:, :2] * er).sum(1))
                                                               / np.mean(np.linalg.norm(ad, axis=1)))}
        out[f"a_{a_target}"] = {"a": a, "rms_net_force": float(np.sqrt((ad ** 2).sum(1).mean())), **rows}
    line = {"workload": "octree_accuracy_n65536", "n": n, "evolution": {"steps": done, "kdk_ms_total": ms,
            "form": "direct, infinite window, correction table"}, "snapshots": out}
    sim.close()
    print(json.dumps(line), flush=True)
    return 0


def run_production(args):
    """The production-shaped run as the workload states it: N = 524,288,
    softening 1:8, LCDM from a = 0.02 to a = 1 in 1000 KDK steps, the learned
    tail with FP32-Kahan near images, and the plain image sum re-checking it
    every 50 steps (a failed check falls back to the plain sum). Per chunk of 50
    steps one JSON line goes to --log (a, t, step time, the momentum drift, the
    check's errors, the form in use); a checkpoint is written every
    --ckpt-every steps to --ckpt, and --resume continues from one. At the end
    the forces of both forms are compared with the FP64 oracle on 4,096
    particles (seed 12345) at the final state."""
    import torch
    from paper_2602_20787_gb300 import ics, steps_cyl as sc
    w = ics.WORKLOADS["production_n524288"]
    d = ics.workload_ics(w)
    n = w.n
    t0, dt = ics.run_schedule(w)
    stream = torch.cuda.current_stream().cuda_stream
    log = open(args.log, "a") if args.log else None
    if args.resume:
        sim = sc.Simulation.resume(args.resume, 0, stream)
        rec = json.load(open(args.resume + ".json"))
    else:
        cfg = sc.Config(n_cut=w.n_cut, n0=w.n0, precision=sc.STEPS_FP32_KAHAN, rho_bar=w.rho_bar, comoving=True,
                        a_start=w.a_start, t_start=t0, check_every=CHECK_EVERY, check_particles=1024, stream=stream)
        sim = sc.Simulation(cfg, d["pos"], d["vel"], d["m"], d["h"])
        rep = sc.steps_cyl_train_surrogate(sim.ctx, sc.steps_cyl_train_cfg_default())
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
        d0 = sim.diagnostics()
        rec = {"done": 0, "fallbacks": 0, "step_ms_total": 0.0, "P0": [float(v) for v in d0[:3]], "Lz0": float(d0[3]),
               "train": {"ms": float(rep[5]), "check_median": float(rep[2]), "check_p999": float(rep[3])},
               "form": "surrogate"}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stop = min(w.nsteps, rec["done"] + (args.steps_limit or w.nsteps))
    while rec["done"] < stop:
        k = min(CHECK_EVERY - rec["done"] % CHECK_EVERY, stop - rec["done"])
        ev0.record()
        fell_back = False
        try:
            sim.step(dt, k)
        except sc.StepsError as e:   # a periodic check dropped the network: the plain sum carries on
            if e.code != sc.STEPS_ESURROGATE_REJECTED:
                raise
            fell_back = True
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        rec["done"] += k
        rec["step_ms_total"] += ms
        if fell_back:
            rec["fallbacks"] += 1
            rec["form"] = "plain"
        dg = sim.diagnostics()
        x, v, a, t = sim.state()
        p = v * a * a
        pscale = float(np.sum(d["m"][:, None] * np.abs(p)))
        chunk = {"step": rec["done"], "a": float(dg[5]), "t": float(dg[6]), "step_ms": ms / k,
                 "pz_drift_over_momentum_scale": abs(float(dg[2]) - rec["P0"][2]) / pscale,
                 "lz_drift_over_scale": abs(float(dg[3]) - rec["Lz0"]) /
                 float(np.sum(d["m"] * np.hypot(x[:, 0], x[:, 1]) * np.linalg.norm(p, axis=1))),
                 "form": rec["form"], "fell_back": fell_back}
        if rec["done"] % CHECK_EVERY == 0 and rec["form"] == "surrogate":
            ck = sc.steps_cyl_check_surrogate(sim.ctx, 1024)
            chunk["check_median"], chunk["check_p999"] = float(ck[0]), float(ck[1])
        if log:
            log.write(json.dumps(chunk) + "\n")
            log.flush()
        rec["last"] = chunk
        if args.ckpt and (rec["done"] % args.ckpt_every == 0 or rec["done"] == stop):
            sim.checkpoint(args.ckpt)
            with open(args.ckpt + ".json", "w") as fh:
                json.dump(rec, fh)
    line = {"workload": "production_run_n524288", "n": n, "n_cut": w.n_cut, "n0": w.n0, "steps_done": rec["done"],
            "steps_total": w.nsteps, "fallbacks": rec["fallbacks"], "form_at_end": rec["form"],
            "mean_step_ms": rec["step_ms_total"] / max(rec["done"], 1), "last": rec.get("last"),
            "train": rec["train"]}
    if rec["done"] >= w.nsteps:
        # both forms against the FP64 oracle at the final state
        import oracle
        oracle.build()
        x, v, a, t = sim.state()
        idx = ics.subsample(n, 4096, seed=12345)
        forms = {"plain": sc.STEPS_TAIL_FULL}
        if rec["form"] == "surrogate":
            forms = {"surrogate": sc.STEPS_TAIL_SURROGATE, "plain": sc.STEPS_TAIL_FULL}
        got = {}
        for name, tail in forms.items():
            sc.steps_cyl_set_tail(sim.ctx, tail)
            got[name] = sim.forces_subset(idx)
        to0 = time.perf_counter()
        ref = (oracle.pair_field(x, d["m"], d["h"], 1.0, 1.0, w.n_cut, idx=idx)
               + oracle.background_field(x[idx], ics.R_SIM, w.n_cut * 1.0, 1.0, w.rho_bar, mode=1)) / a ** 3
        line["oracle_seconds"] = time.perf_counter() - to0
        line["a_end"] = a
        line["error_vs_oracle"] = {k: _err(g, ref) for k, g in got.items()}
    sim.close()
    if log:
        log.close()
    print(json.dumps(line), flush=True)
    return 0


def run_workload(args):
    import torch
    from paper_2602_20787_gb300 import ics, steps_cyl as sc
    if args.workload == "production_run":
        return run_production(args)
    if args.workload == "octree_accuracy_n65536":
        return run_octree_accuracy(args)
    if args.workload == "octree_r3_n1048576":
        return run_octree_r3(args)
    if args.workload in ("r3_n65536", "glass_n65536"):
        return run_r3_or_glass(args)
    if args.workload in ("octree_n65536", "octree_n524288"):
        return run_octree(args)
    if args.workload == "inf_n65536":
        return run_inf(args)
    if args.workload == "table1_n65536":
        return run_table1(args)
    w = ics.WORKLOADS[args.workload]
    d = ics.workload_ics(w)
    n = w.n
    pairs = n * (n - 1.0)
    props = torch.cuda.get_device_properties(0)
    peak = props.multi_processor_count * MUFU_RSQRT_PER_SM_CLK * 2070e6
    line = {"workload": w.name, "n": n, "n_cut": w.n_cut, "roofline_peak_pair_images_per_s": peak}
    idx = ics.subsample(n, 4096 if w.name.startswith("precision") else 256, seed=12345)
    reps = 1 if n > 300000 else 2
    sim = _ctx_for(sc, torch, w, d, sc.STEPS_FP32_KAHAN, check_particles=1024,
                   check_every=10 if w.name.startswith("production") else 50)
    a32, ms32 = _timed_forces(sc, torch, sim, reps)
    ev32 = sc.steps_cyl_last_eval(sim.ctx)
    line["fp32_kahan"] = {"pair_ms": ms32, "pair_images_per_s": pairs * 2 * w.n_cut / (ms32 * 1e-3),
                          "symmetric": ev32["symmetric"],
                          "roofline_frac": ev32["pairs_evaluated"] * 2 * w.n_cut / (ms32 * 1e-3) / peak}
    sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP64)
    a64 = sim.forces_subset(idx)
    ms64 = sc.steps_cyl_last_timing(sim.ctx)[1]
    line["fp64_subset"] = {"i_sample": int(idx.size), "pair_ms": ms64,
                           "pair_images_per_s": idx.size * (n - 1.0) * 2 * w.n_cut / (ms64 * 1e-3)}
    sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP32_KAHAN)
    line["fp32_kahan"]["error_vs_fp64"] = _err(a32[idx], a64)
    if w.name.startswith("precision"):
        sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP32_PLAIN)
        ap, msp = _timed_forces(sc, torch, sim, reps)
        line["fp32_plain"] = {"pair_ms": msp, "pair_images_per_s": pairs * 2 * w.n_cut / (msp * 1e-3),
                              "error_vs_fp64": _err(ap[idx], a64)}
        # every form against the FP64 oracle itself on the same 4,096 particles
        # (pair field of eq. ComovingEquationsOfMotionCylindrical against all j,
        # plus the background of eq. F_horiz), in the library's units (1 / a^3)
        import oracle
        oracle.build()
        to0 = time.perf_counter()
        o_pair = oracle.pair_field(d["pos"], d["m"], d["h"], 1.0, 1.0, w.n_cut, idx=idx)
        o_bg = oracle.background_field(d["pos"][idx], ics.R_SIM, w.n_cut * 1.0, 1.0, w.rho_bar, mode=1)
        oracle_s = time.perf_counter() - to0
        inv_a3 = 1.0 / w.a_start ** 3
        o_tot, o_pair = (o_pair + o_bg) * inv_a3, o_pair * inv_a3
        line["oracle_reference"] = {
            "what": f"FP64 oracle pair field + background of {idx.size} particles (seed 12345) against all {n} j, "
                    f"{2 * w.n_cut} images per pair", "cores": oracle.num_threads(), "seconds": oracle_s}
        line["fp64_subset"]["error_vs_oracle"] = _err(a64, o_tot)
        for key, a in (("fp32_kahan", a32[idx]), ("fp32_plain", ap[idx])):
            line[key]["error_vs_oracle"] = _err(a, o_tot)
            r = np.linalg.norm(a - o_tot, axis=1) / np.linalg.norm(o_pair, axis=1)
            line[key]["error_vs_oracle_over_pair_term"] = {"median": float(np.median(r)),
                                                           "p999": float(np.quantile(r, 0.999)),
                                                           "max": float(r.max())}
        # pair-only errors: the same differences over the FP64 pair term alone (a context without the
        # background, whose FP64 subset gives the pair term; the background itself is FP64 in every form)
        nobg = _ctx_for(sc, torch, w, d, sc.STEPS_FP32_PLAIN, background=sc.STEPS_BG_OFF)
        sc.steps_cyl_set_precision(nobg.ctx, sc.STEPS_FP64)
        p64 = nobg.forces_subset(idx)
        nobg.close()
        for key, a in (("fp32_kahan", a32), ("fp32_plain", ap)):
            r = np.linalg.norm(a[idx] - a64, axis=1) / np.linalg.norm(p64, axis=1)
            line[key]["error_vs_fp64_pair_only"] = {"median": float(np.median(r)),
                                                    "p999": float(np.quantile(r, 0.999)), "max": float(r.max())}
    if w.name.startswith("surrogate") or w.name.startswith("production"):
        sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP32_KAHAN)
        rep = sc.steps_cyl_train_surrogate(sim.ctx, sc.steps_cyl_train_cfg_default())
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
        asg, mss = _timed_forces(sc, torch, sim, reps + 1)
        line["surrogate"] = {
            "train_ms": rep[5], "train_heldout_rms": rep[1], "check_median": rep[2], "check_p999": rep[3],
            "pair_ms": mss, "equivalent_pair_images_per_s": pairs * 2 * w.n_cut / (mss * 1e-3),
            "executed_near_images_per_pair": 2 * w.n0 + 1, "speedup_vs_fp32_plain_sum": ms32 / mss,
            "error_vs_fp64": _err(asg[idx], a64)}
        ev = sc.steps_cyl_last_eval(sim.ctx)
        line["surrogate"]["roofline"] = surrogate_roofline(props.multi_processor_count, 2070.0, w.n0,
                                                           ev["pairs_evaluated"], mss * 1e-3, ev["symmetric"],
                                                           headline=False)
        # correction-table tail: near images exact, tail from the GPU-built table
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_FULL)
        nx, ny = 257, 33
        rt = sc.steps_cyl_build_tail_table(sim.ctx, nx, ny)
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
        atb, mst = _timed_forces(sc, torch, sim, reps + 1)
        ev_t = sc.steps_cyl_last_eval(sim.ctx)
        mufu_t = (2 * w.n0 + 1) + 4 + 2 + 1   # near images, base rsqrt/rcp, the dR rsqrt
        peak_t = props.multi_processor_count * 2070e6 * MUFU_RSQRT_PER_SM_CLK / mufu_t
        import oracle
        dR_t = max(2.2 * float(np.hypot(d["pos"][:, 0], d["pos"][:, 1]).max()), 1.0)
        tcfg = oracle.make_table_cfg(w.n_cut, w.n0, nx, ny, dR_t)
        ttab = oracle.tail_table_build(tcfg)
        line["table_cpu_baseline"] = oracle_rate(
            lambda ix: oracle.pair_field_table(d["pos"], d["m"], d["h"], 1.0, 1.0, ttab, tcfg, idx=ix), n, n - 1.0,
            "pair interactions/s", f"FP64 table form, all {n} j")
        sp = ics.random_surrogate_params(5, dR_t)
        scfg = oracle.make_surr_cfg(w.n_cut, w.n0, dR_t, (0.0, 0.0), (0.05, 0.05))
        w16 = sp[:1250].astype(np.float16).astype(np.float64)
        line["surrogate_cpu_baseline"] = oracle_rate(
            lambda ix: oracle.pair_field_surrogate(d["pos"], d["m"], d["h"], 1.0, 1.0, w16, scfg, idx=ix), n,
            n - 1.0, "pair interactions/s", f"FP64 surrogate form (seeded network), all {n} j")
        line["table"] = {
            "nx": nx, "ny": ny, "build_ms": rt[3], "check_median": rt[0], "check_p999": rt[1], "pair_ms": mst,
            "equivalent_pair_images_per_s": pairs * 2 * w.n_cut / (mst * 1e-3),
            "speedup_vs_fp32_plain_sum": ms32 / mst, "speedup_vs_surrogate": mss / mst,
            "error_vs_fp64": _err(atb[idx], a64),
            "roofline": {"bound": "mufu", "mufu_ops_per_pair": mufu_t, "peak_pairs_per_s": peak_t,
                         "achieved_pairs_evaluated_per_s": ev_t["pairs_evaluated"] / (mst * 1e-3),
                         "frac": ev_t["pairs_evaluated"] / (mst * 1e-3) / peak_t, "symmetric": ev_t["symmetric"]}}
        # the same table read with TSC weights (Sect. 2.3 names CIC and TSC)
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_FULL)
        sc.steps_cyl_set_table_read(sim.ctx, sc.STEPS_TABLE_READ_TSC)
        rq = sc.steps_cyl_build_tail_table(sim.ctx, nx, ny)
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_TABLE)
        atq, msq = _timed_forces(sc, torch, sim, reps + 1)
        line["table_tsc"] = {"check_median": rq[0], "check_p999": rq[1], "pair_ms": msq,
                             "equivalent_pair_images_per_s": pairs * 2 * w.n_cut / (msq * 1e-3),
                             "error_vs_fp64": _err(atq[idx], a64), "cost_vs_cic": msq / mst}
        sc.steps_cyl_set_table_read(sim.ctx, sc.STEPS_TABLE_READ_CIC)
        sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_FULL)
    if w.name.startswith("production") or w.name.startswith("plain_small") or w.name.startswith("lcdm"):
        steps = min(args.steps, w.nsteps) if w.nsteps else args.steps
        t0, dt = ics.run_schedule(w)
        sc.steps_cyl_set_precision(sim.ctx, sc.STEPS_FP32_KAHAN)
        if w.name.startswith("production"):
            sc.steps_cyl_set_tail(sim.ctx, sc.STEPS_TAIL_SURROGATE)
        d0 = sim.diagnostics()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        sim.step(dt, steps)
        ev1.record()
        torch.cuda.synchronize()
        d1 = sim.diagnostics()
        # momentum scale: total mass times the rms canonical velocity a^2 |dx/dt|
        pscale = d1[5] ** 2 * math.sqrt(2.0 * d1[4] * d1[7]) if d1[4] > 0 else 1.0
        line["kdk"] = {"steps": steps, "dt": dt, "step_ms": ev0.elapsed_time(ev1) / steps, "a_end": d1[5],
                       "pz_drift_over_momentum_scale": abs(d1[2] - d0[2]) / pscale,
                       "lz_drift_abs": abs(d1[3] - d0[3]),
                       "tail": "surrogate" if w.name.startswith("production") else "full"}
    sim.close()
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=None, help="run another workload's measurement (one JSON line)")
    ap.add_argument("--log", default=None, help="production_run: per-chunk JSON lines")
    ap.add_argument("--ckpt", default=None, help="production_run: checkpoint path")
    ap.add_argument("--ckpt-every", type=int, default=250, help="production_run: steps between checkpoints")
    ap.add_argument("--resume", default=None, help="production_run: continue from this checkpoint")
    ap.add_argument("--steps-limit", type=int, default=0, help="production_run: stop after this many steps")
    args = ap.parse_args()
    if args.workload:
        sys.exit(run_workload(args))
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    sys.exit(run(args))


if __name__ == "__main__":
    main()
