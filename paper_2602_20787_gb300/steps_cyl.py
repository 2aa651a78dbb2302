"""Python binding of the C ABI in ``include/steps_cyl.h`` (ctypes).

Argument marshalling only: every step of the hot path runs in the CUDA library
``libsteps_cyl.so`` built in-tree by ``paper_2602_20787_gb300.build``. If that
library is missing or cannot be loaded, every call raises: there is no CPU
fallback. Arrays may be CUDA torch tensors (device pointers are passed straight
through), CPU torch tensors or numpy arrays (host pointers; the library copies).
All arrays are float64 (indices int64) and contiguous.
"""
from __future__ import annotations

import ctypes
import dataclasses
import json
import math
import os
import time

import numpy as np

from . import build as _build

STEPS_OK = 0
STEPS_EINVAL = -1
STEPS_ECUDA = -2
STEPS_ENOMEM = -3
STEPS_EDEVICE = -4
STEPS_ESURROGATE_REJECTED = -5
STEPS_ENOSURROGATE = -6

STEPS_FP64, STEPS_FP32_KAHAN, STEPS_FP32_PLAIN = 0, 1, 2
STEPS_TAIL_FULL, STEPS_TAIL_SURROGATE, STEPS_TAIL_TABLE = 0, 1, 2
STEPS_TABLE_READ_CIC, STEPS_TABLE_READ_TSC = 0, 1
STEPS_BG_OFF, STEPS_BG_FINITE, STEPS_BG_INFINITE, STEPS_BG_SPHERE = 0, 1, 2, 3
STEPS_TOPO_S1R2, STEPS_TOPO_R3 = 0, 1
STEPS_FORCE_DIRECT, STEPS_FORCE_OCTREE = 0, 1

_EXPORTS = [
    "steps_cyl_params_default", "steps_cyl_init", "steps_cyl_forces", "steps_cyl_forces_subset",
    "steps_cyl_kdk_step", "steps_cyl_get_state", "steps_cyl_set_state", "steps_cyl_set_precision",
    "steps_cyl_diagnostics", "steps_cyl_last_timing", "steps_cyl_free", "steps_cyl_strerror",
    "steps_cyl_last_error", "steps_cyl_pair_accel_noalloc", "steps_cyl_train_cfg_default", "steps_cyl_tail_sums",
    "steps_cyl_mlp_loss_grad", "steps_cyl_train_surrogate", "steps_cyl_set_surrogate", "steps_cyl_get_surrogate",
    "steps_cyl_set_tail", "steps_cyl_check_surrogate", "steps_cyl_checkpoint", "steps_cyl_resume",
    "steps_cyl_build_tail_table", "steps_cyl_build_tail_table_ewald", "steps_cyl_get_tail_table",
    "steps_cyl_check_tail", "steps_cyl_set_table_read",
    "steps_cyl_tree_frame", "steps_cyl_tree_frame_r3", "steps_cyl_tree_stats", "steps_cyl_tree_calibrate",
    "steps_cyl_tree_set_radial", "steps_cyl_shard", "steps_cyl_shard_drift", "steps_cyl_shard_kick",
    "steps_cyl_last_eval", "steps_cyl_shard_mode", "steps_cyl_shard_force", "steps_cyl_shard_finish",
    "steps_cyl_surrogate_lanes",
]

STEPS_SURR_NW = 1250
STEPS_SURR_NPARAM = 1255
STEPS_SURR_LANE_WORDS = 44

# size limit of the allocation-free entry point (include/steps_cyl.h)
STEPS_NOALLOC_MAX_N = 65536


class StepsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class Params(ctypes.Structure):
    """Mirror of ``steps_cyl_params``."""
    _fields_ = [
        ("G", ctypes.c_double), ("L", ctypes.c_double), ("R_sim", ctypes.c_double), ("rho_bar", ctypes.c_double),
        ("n_cut", ctypes.c_int32), ("n0", ctypes.c_int32), ("precision", ctypes.c_int32), ("tail", ctypes.c_int32),
        ("background", ctypes.c_int32), ("comoving", ctypes.c_int32),
        ("H0", ctypes.c_double), ("Omega_m", ctypes.c_double), ("Omega_r", ctypes.c_double),
        ("Omega_L", ctypes.c_double), ("w0", ctypes.c_double), ("wa", ctypes.c_double),
        ("a_start", ctypes.c_double), ("t_start", ctypes.c_double),
        ("device", ctypes.c_int32), ("reorder_every", ctypes.c_int32), ("check_every", ctypes.c_int32),
        ("check_particles", ctypes.c_int32), ("topology", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("force", ctypes.c_int32), ("leaf_size", ctypes.c_int32), ("theta", ctypes.c_double),
        ("tree_seed", ctypes.c_uint64),
    ]


class TrainCfg(ctypes.Structure):
    """Mirror of ``steps_cyl_train_cfg``."""
    _fields_ = [
        ("n_samples", ctypes.c_int64), ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_double),
        ("dR_max", ctypes.c_double), ("seed", ctypes.c_uint64), ("err_median", ctypes.c_double),
        ("err_p999", ctypes.c_double), ("check_particles", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library; raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    checked = os.environ.get("STEPS_CYL_INDEX_CHECKED") == "1"   # the index-checked test build
    path = _build.LIB_CHECKED if checked else _build.LIB
    if build_if_missing:
        path = _build.build(checked=checked)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run paper_2602_20787_gb300.build.build()")
    L = ctypes.CDLL(path)
    p, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.steps_cyl_params_default.argtypes = [ctypes.POINTER(Params)]
    L.steps_cyl_init.argtypes = [ctypes.POINTER(p), ctypes.POINTER(Params), i64] + [p] * 8
    L.steps_cyl_forces.argtypes = [p, p, p, p]
    L.steps_cyl_forces_subset.argtypes = [p, i64, p, p, p, p]
    L.steps_cyl_kdk_step.argtypes = [p, d, i32]
    L.steps_cyl_get_state.argtypes = [p] * 9
    L.steps_cyl_set_state.argtypes = [p] * 7
    L.steps_cyl_set_precision.argtypes = [p, i32]
    L.steps_cyl_diagnostics.argtypes = [p, p]
    L.steps_cyl_last_timing.argtypes = [p, p, p]
    L.steps_cyl_last_eval.argtypes = [p, p]
    L.steps_cyl_free.argtypes = [p]
    L.steps_cyl_strerror.argtypes = [ctypes.c_int]
    L.steps_cyl_strerror.restype = ctypes.c_char_p
    L.steps_cyl_last_error.argtypes = []
    L.steps_cyl_last_error.restype = ctypes.c_char_p
    L.steps_cyl_pair_accel_noalloc.argtypes = [i64, p, p, p, p, p, d, d, i32, i32, p, p, p, p]
    L.steps_cyl_train_cfg_default.argtypes = [ctypes.POINTER(TrainCfg)]
    L.steps_cyl_tail_sums.argtypes = [i64, p, i32, i32, p, p]
    L.steps_cyl_mlp_loss_grad.argtypes = [i64, p, p, p, p, p, p]
    L.steps_cyl_train_surrogate.argtypes = [p, ctypes.POINTER(TrainCfg), p]
    L.steps_cyl_set_surrogate.argtypes = [p, p, d, d, p]
    L.steps_cyl_get_surrogate.argtypes = [p, p]
    L.steps_cyl_surrogate_lanes.argtypes = [p, p, p]
    L.steps_cyl_set_tail.argtypes = [p, i32]
    L.steps_cyl_check_surrogate.argtypes = [p, i32, p]
    L.steps_cyl_build_tail_table.argtypes = [p, i32, i32, d, d, d, i32, p]
    L.steps_cyl_build_tail_table_ewald.argtypes = [p, i32, i32, d, d, i32, i32, p]
    L.steps_cyl_set_table_read.argtypes = [p, i32]
    L.steps_cyl_get_tail_table.argtypes = [p, p, p, p, p]
    L.steps_cyl_check_tail.argtypes = [p, i32, i32, p]
    L.steps_cyl_checkpoint.argtypes = [p, ctypes.c_char_p]
    L.steps_cyl_resume.argtypes = [ctypes.POINTER(p), ctypes.c_char_p, i32, p]
    L.steps_cyl_tree_frame.argtypes = [p, d, d]
    L.steps_cyl_tree_frame_r3.argtypes = [p, p]
    L.steps_cyl_tree_stats.argtypes = [p, p]
    L.steps_cyl_tree_calibrate.argtypes = [p, i32, i32, i32, p, p, p, p]
    L.steps_cyl_tree_set_radial.argtypes = [p, p, i32, d]
    L.steps_cyl_shard.argtypes = [p, i32, i32, p]
    L.steps_cyl_shard_drift.argtypes = [p, d, p]
    L.steps_cyl_shard_kick.argtypes = [p, p]
    L.steps_cyl_shard_mode.argtypes = [p, p, p]
    L.steps_cyl_shard_force.argtypes = [p, p, p]
    L.steps_cyl_shard_finish.argtypes = [p, p]
    for name in _EXPORTS:
        fn = getattr(L, name)
        if fn.restype is None or fn.restype is ctypes.c_int:
            fn.restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != STEPS_OK:
        L = load(False)
        msg = (L.steps_cyl_last_error() or b"").decode() or L.steps_cyl_strerror(rc).decode()
        raise StepsError(rc, msg)


def _ptr(a):
    """Raw data pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data_as(ctypes.c_void_p)
    raise TypeError(f"unsupported array type {type(a)}")


def _check_f64(*arrs):
    for a in arrs:
        if a is None:
            continue
        dt = getattr(a, "dtype", None)
        if str(dt) not in ("float64", "torch.float64"):
            raise TypeError(f"float64 arrays required, got {dt}")


@dataclasses.dataclass
class Config:
    G: float = 1.0
    L: float = 1.0
    R_sim: float = 0.5 * math.tan(0.45 * math.pi)
    rho_bar: float = 0.0
    n_cut: int = 16
    n0: int = 4
    precision: int = STEPS_FP32_KAHAN
    tail: int = STEPS_TAIL_FULL
    background: int = STEPS_BG_FINITE
    comoving: bool = False
    H0: float = 1.0
    Omega_m: float = 0.3
    Omega_r: float = 0.0
    Omega_L: float = 0.7
    w0: float = -1.0
    wa: float = 0.0
    a_start: float = 1.0
    t_start: float = 0.0
    device: int = 0
    reorder_every: int = 32
    check_every: int = 50
    check_particles: int = 1024
    topology: int = STEPS_TOPO_S1R2
    force: int = STEPS_FORCE_DIRECT
    leaf_size: int = 16
    theta: float = 0.5
    tree_seed: int = 1
    stream: int = 0  # cudaStream_t as an integer (torch.cuda.Stream.cuda_stream), 0 = default

    def to_c(self) -> Params:
        p = Params()
        load().steps_cyl_params_default(ctypes.byref(p))
        for f in dataclasses.fields(self):
            if f.name == "stream":
                p.stream = ctypes.c_void_p(self.stream or None)
            elif f.name == "comoving":
                p.comoving = 1 if self.comoving else 0
            else:
                setattr(p, f.name, getattr(self, f.name))
        return p


def steps_cyl_params_default() -> Params:
    p = Params()
    _check(load().steps_cyl_params_default(ctypes.byref(p)))
    return p


def steps_cyl_init(cfg, n, x, y, z, vx, vy, vz, m, h) -> ctypes.c_void_p:
    _check_f64(x, y, z, vx, vy, vz, m, h)
    p = cfg.to_c() if isinstance(cfg, Config) else cfg
    ctx = ctypes.c_void_p()
    _check(load().steps_cyl_init(ctypes.byref(ctx), ctypes.byref(p), int(n), _ptr(x), _ptr(y), _ptr(z), _ptr(vx),
                                 _ptr(vy), _ptr(vz), _ptr(m), _ptr(h)))
    return ctx


def steps_cyl_forces(ctx, ax, ay, az):
    _check_f64(ax, ay, az)
    _check(load().steps_cyl_forces(ctx, _ptr(ax), _ptr(ay), _ptr(az)))


def steps_cyl_forces_subset(ctx, idx, ax, ay, az):
    _check_f64(ax, ay, az)
    _check(load().steps_cyl_forces_subset(ctx, int(len(idx)), _ptr(idx), _ptr(ax), _ptr(ay), _ptr(az)))


def steps_cyl_kdk_step(ctx, dt: float, nsteps: int):
    _check(load().steps_cyl_kdk_step(ctx, float(dt), int(nsteps)))


def steps_cyl_get_state(ctx, x=None, y=None, z=None, vx=None, vy=None, vz=None):
    _check_f64(x, y, z, vx, vy, vz)
    a, t = ctypes.c_double(), ctypes.c_double()
    _check(load().steps_cyl_get_state(ctx, _ptr(x), _ptr(y), _ptr(z), _ptr(vx), _ptr(vy), _ptr(vz),
                                      ctypes.byref(a), ctypes.byref(t)))
    return a.value, t.value


def steps_cyl_set_state(ctx, x, y, z, vx, vy, vz):
    _check_f64(x, y, z, vx, vy, vz)
    _check(load().steps_cyl_set_state(ctx, _ptr(x), _ptr(y), _ptr(z), _ptr(vx), _ptr(vy), _ptr(vz)))


def steps_cyl_set_precision(ctx, precision: int):
    _check(load().steps_cyl_set_precision(ctx, int(precision)))


def steps_cyl_diagnostics(ctx) -> np.ndarray:
    out = np.zeros(8)
    _check(load().steps_cyl_diagnostics(ctx, _ptr(out)))
    return out


def steps_cyl_last_timing(ctx):
    imgs, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().steps_cyl_last_timing(ctx, ctypes.byref(imgs), ctypes.byref(ms)))
    return imgs.value, ms.value


def steps_cyl_last_eval(ctx) -> dict:
    """The last direct force evaluation: pair-images delivered, pairs the
    kernel evaluated, its device ms, whether it was a symmetric kernel, and
    whether that kernel took the modelled tails' straight run."""
    out = np.zeros(4)
    _check(load().steps_cyl_last_eval(ctx, _ptr(out)))
    return {"pair_images": float(out[0]), "pairs_evaluated": float(out[1]), "pair_ms": float(out[2]),
            "symmetric": bool(out[3]), "straight_run": out[3] == 2.0}


def steps_cyl_free(ctx):
    if ctx:
        _check(load().steps_cyl_free(ctx))


def steps_cyl_pair_accel_noalloc(x, y, z, m, h, G, L, n_cut, precision, ax, ay, az, stream=0):
    """Pair accelerations with no device allocation, for callers that may not
    allocate device memory (see include/steps_cyl.h for the contract, its
    scratch limit and why concurrent calls must be serialised). Every array is a
    contiguous float64 CUDA tensor of the current device with the same length n;
    the outputs ax, ay, az are written in place. Anything else raises before the
    library is called."""
    import torch
    arrs = (x, y, z, m, h, ax, ay, az)
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None
    for a in arrs:
        if not isinstance(a, torch.Tensor) or not a.is_cuda:
            raise StepsError(STEPS_EINVAL, "every array must be a CUDA tensor")
        if a.device.index != dev:
            raise StepsError(STEPS_EINVAL, f"arrays must live on the current device cuda:{dev}")
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise StepsError(STEPS_EINVAL, "arrays must be contiguous float64")
    n = int(x.numel())
    if any(int(a.numel()) != n for a in arrs):
        raise StepsError(STEPS_EINVAL, "all eight arrays must have the same length")
    if n > STEPS_NOALLOC_MAX_N:
        raise StepsError(STEPS_EINVAL, f"n = {n} exceeds STEPS_NOALLOC_MAX_N = {STEPS_NOALLOC_MAX_N}")
    rc = load().steps_cyl_pair_accel_noalloc(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h), float(G), float(L),
                                             int(n_cut), int(precision), _ptr(ax), _ptr(ay), _ptr(az),
                                             ctypes.c_void_p(stream or None))
    if rc != STEPS_OK:
        raise StepsError(rc, "steps_cyl_pair_accel_noalloc rejected its arguments or failed to launch")


def steps_cyl_shard(ctx, rank: int, world: int):
    """Make the context shard `rank` of `world` (row sharding): returns the
    owned internal rows (k0, k1) and chunk, the rows per rank of an exchange."""
    rows = np.zeros(3, dtype=np.int64)
    _check(load().steps_cyl_shard(ctx, int(rank), int(world), _ptr(rows)))
    return int(rows[0]), int(rows[1]), int(rows[2])


def _exchange_buffer(buf, what):
    if not hasattr(buf, "is_cuda") or not buf.is_cuda or str(buf.dtype) != "torch.float32":
        raise StepsError(STEPS_EINVAL, f"{what} must be a float32 CUDA tensor")
    return _ptr(buf)


def steps_cyl_shard_drift(ctx, dt: float, send):
    """First half of a sharded KDK step; the owned packed rows go to send
    (float32 CUDA tensor of chunk x 8)."""
    _check(load().steps_cyl_shard_drift(ctx, float(dt), _exchange_buffer(send, "send")))


def steps_cyl_shard_kick(ctx, recv):
    """Second half of a sharded KDK step from the gathered rows (float32 CUDA
    tensor of world x chunk x 8, rank order)."""
    _check(load().steps_cyl_shard_kick(ctx, _exchange_buffer(recv, "recv")))


def steps_cyl_shard_mode(ctx):
    """(symmetric, sums_len): whether the sharded context offers the symmetric
    two-exchange step, and the int64 length of its sums buffer."""
    sym = ctypes.c_int32()
    ln = ctypes.c_int64()
    _check(load().steps_cyl_shard_mode(ctx, ctypes.byref(sym), ctypes.byref(ln)))
    return bool(sym.value), int(ln.value)


def _int64_cuda(buf, what):
    if not hasattr(buf, "is_cuda") or not buf.is_cuda or str(buf.dtype) != "torch.int64":
        raise StepsError(STEPS_EINVAL, f"{what} must be an int64 CUDA tensor")
    return _ptr(buf)


def steps_cyl_shard_force(ctx, recv, sums):
    """This rank's share of the unordered pairs into sums (int64 CUDA tensor of
    world x 3 x chunk), from the gathered rows recv."""
    _check(load().steps_cyl_shard_force(ctx, _exchange_buffer(recv, "recv"), _int64_cuda(sums, "sums")))


def steps_cyl_shard_finish(ctx, own):
    """Finish the symmetric sharded step from this rank's reduced sums (int64
    CUDA tensor of 3 x chunk)."""
    _check(load().steps_cyl_shard_finish(ctx, _int64_cuda(own, "own")))


def steps_cyl_train_cfg_default(**overrides) -> TrainCfg:
    cfg = TrainCfg()
    _check(load().steps_cyl_train_cfg_default(ctypes.byref(cfg)))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def steps_cyl_tail_sums(samples, n_cut: int, n0: int, stream=0) -> np.ndarray:
    """Exact FP64 far-image tail sums on the GPU for samples (ns, 3) = (dR, dz, h) in units of L."""
    smp = np.ascontiguousarray(samples, dtype=np.float64)
    out = np.zeros((smp.shape[0], 2))
    _check(load().steps_cyl_tail_sums(smp.shape[0], _ptr(smp), int(n_cut), int(n0), _ptr(out),
                                      ctypes.c_void_p(stream or None)))
    return out


def steps_cyl_mlp_loss_grad(w, u, t, stream=0):
    """FP32 forward + backward of the surrogate network on the GPU: (loss, grad)."""
    w = np.ascontiguousarray(w, dtype=np.float32)
    u = np.ascontiguousarray(u, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    grad = np.zeros(STEPS_SURR_NW, dtype=np.float32)
    _check(load().steps_cyl_mlp_loss_grad(u.shape[0], _ptr(w), _ptr(u), _ptr(t), _ptr(loss), _ptr(grad),
                                          ctypes.c_void_p(stream or None)))
    return float(loss[0]), grad


def steps_cyl_train_surrogate(ctx, cfg: TrainCfg) -> np.ndarray:
    """Train and check the context's surrogate; returns the 8-entry report.
    Raises StepsError (code STEPS_ESURROGATE_REJECTED) when the check fails."""
    rep = np.zeros(8)
    rc = load().steps_cyl_train_surrogate(ctx, ctypes.byref(cfg), _ptr(rep))
    if rc == STEPS_ESURROGATE_REJECTED:
        err = StepsError(rc, (load().steps_cyl_last_error() or b"").decode())
        err.report = rep
        raise err
    _check(rc)
    return rep


def steps_cyl_set_surrogate(ctx, params, err_median=1e-5, err_p999=1e-3) -> np.ndarray:
    p = np.ascontiguousarray(params, dtype=np.float32)
    rep = np.zeros(4)
    rc = load().steps_cyl_set_surrogate(ctx, _ptr(p), float(err_median), float(err_p999), _ptr(rep))
    if rc == STEPS_ESURROGATE_REJECTED:
        err = StepsError(rc, (load().steps_cyl_last_error() or b"").decode())
        err.report = rep
        raise err
    _check(rc)
    return rep


def steps_cyl_get_surrogate(ctx) -> np.ndarray:
    out = np.zeros(STEPS_SURR_NPARAM, dtype=np.float32)
    _check(load().steps_cyl_get_surrogate(ctx, _ptr(out)))
    return out


def steps_cyl_surrogate_lanes(params):
    """The network's per-lane tensor-core operands as the kernels stage them
    (host only): (lanes uint32 [32][STEPS_SURR_LANE_WORDS], shift float32 [2])."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.shape != (STEPS_SURR_NPARAM,):
        raise StepsError(STEPS_EINVAL, f"params must hold {STEPS_SURR_NPARAM} floats")
    lanes = np.zeros((32, STEPS_SURR_LANE_WORDS), dtype=np.uint32)
    shift = np.zeros(2, dtype=np.float32)
    _check(load().steps_cyl_surrogate_lanes(_ptr(p), _ptr(lanes), _ptr(shift)))
    return lanes, shift


def steps_cyl_set_tail(ctx, tail: int):
    _check(load().steps_cyl_set_tail(ctx, int(tail)))


def steps_cyl_check_surrogate(ctx, check_particles: int = 1024) -> np.ndarray:
    rep = np.zeros(4)
    _check(load().steps_cyl_check_surrogate(ctx, int(check_particles), _ptr(rep)))
    return rep


def steps_cyl_build_tail_table(ctx, nx: int = 257, ny: int = 33, dR_max: float = 0.0, err_median: float = 1e-5,
                               err_p999: float = 1e-3, check_particles: int = 1024) -> np.ndarray:
    """Build and check the correction-table tail; returns the report (median,
    p99.9, accepted, build ms). Raises StepsError when the check rejects it."""
    rep = np.zeros(4)
    _check(load().steps_cyl_build_tail_table(ctx, int(nx), int(ny), float(dR_max), float(err_median),
                                             float(err_p999), int(check_particles), _ptr(rep)))
    return rep


def steps_cyl_build_tail_table_ewald(ctx, nx: int = 144, ny: int = 128, dR_max: float = 0.0, alpha: float = 1.0,
                                     nmax: int = 5, mmax: int = 12) -> np.ndarray:
    """Build the infinite window's table by the Ewald summation of the line;
    returns (largest node difference to the direct construction, largest node
    magnitude, Ewald build ms, direct build ms)."""
    rep = np.zeros(4)
    _check(load().steps_cyl_build_tail_table_ewald(ctx, int(nx), int(ny), float(dR_max), float(alpha), int(nmax),
                                                   int(mmax), _ptr(rep)))
    return rep


def steps_cyl_set_table_read(ctx, read: int):
    """STEPS_TABLE_READ_CIC or STEPS_TABLE_READ_TSC for the next table build."""
    _check(load().steps_cyl_set_table_read(ctx, int(read)))


def steps_cyl_get_tail_table(ctx):
    """The table as (ny, nx, 2) float32 residuals, and its dR_max."""
    nx, ny, dm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(load().steps_cyl_get_tail_table(ctx, None, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(dm)))
    out = np.zeros((ny.value, nx.value, 2), dtype=np.float32)
    _check(load().steps_cyl_get_tail_table(ctx, _ptr(out), None, None, None))
    return out, dm.value


def steps_cyl_check_tail(ctx, tail: int, check_particles: int = 1024) -> np.ndarray:
    rep = np.zeros(4)
    _check(load().steps_cyl_check_tail(ctx, int(tail), int(check_particles), _ptr(rep)))
    return rep


def steps_cyl_tree_frame(ctx, zeta: float, phi: float):
    """Fix the octree frame (shift zeta along the axis, rotation phi); zeta < 0: random per evaluation."""
    _check(load().steps_cyl_tree_frame(ctx, float(zeta), float(phi)))


def steps_cyl_tree_frame_r3(ctx, centre=None, axis=None, angle: float = 0.0):
    """R^3: fix the octree frame (domain centre, unit rotation axis, angle); no centre: random per evaluation."""
    if centre is None:
        _check(load().steps_cyl_tree_frame_r3(ctx, None))
        return
    f = np.ascontiguousarray(list(centre) + list(axis) + [angle], dtype=np.float64)
    _check(load().steps_cyl_tree_frame_r3(ctx, _ptr(f)))


def steps_cyl_tree_stats(ctx) -> dict:
    out = np.zeros(6)
    _check(load().steps_cyl_tree_stats(ctx, _ptr(out)))
    return {"nodes": int(out[0]), "depth": int(out[1]), "interactions": float(out[2]), "build_ms": float(out[3]),
            "walk_ms": float(out[4]), "evaluations": int(out[5])}


def steps_cyl_tree_calibrate(ctx, n_frames: int, n_bins: int = 64, n_sample: int = 4096, frames=None, sample=None):
    """Radial calibration of the octree; returns (table of n_bins means, rmax)."""
    fr = None if frames is None else np.ascontiguousarray(frames, dtype=np.float64).reshape(-1)
    sm = None if sample is None else np.ascontiguousarray(sample, dtype=np.int64)
    if sm is not None and sm.shape[0] < n_sample:
        raise ValueError("sample holds fewer than n_sample indices")
    tab = np.zeros(max(int(n_bins), 1))
    rmax = ctypes.c_double()
    _check(load().steps_cyl_tree_calibrate(ctx, int(n_frames), int(n_bins), int(n_sample), _ptr(fr), _ptr(sm),
                                           _ptr(tab), ctypes.byref(rmax)))
    return tab, rmax.value


def steps_cyl_tree_set_radial(ctx, table, rmax: float):
    """Install a radial correction table (from steps_cyl_tree_calibrate, possibly of another context)."""
    tab = np.ascontiguousarray(table, dtype=np.float64).reshape(-1)
    _check(load().steps_cyl_tree_set_radial(ctx, _ptr(tab), int(tab.shape[0]), float(rmax)))


def steps_cyl_checkpoint(ctx, path: str):
    _check(load().steps_cyl_checkpoint(ctx, os.fsencode(path)))


def _ckpt_n(path: str) -> int:
    """Particle count stored in a checkpoint header (after magic, version, size, params)."""
    off = 8 + 4 + 4 + ctypes.sizeof(Params)
    with open(path, "rb") as fh:
        fh.seek(off)
        return int(np.frombuffer(fh.read(8), dtype=np.int64)[0])


def steps_cyl_resume(path: str, device: int = 0, stream: int = 0):
    ctx = ctypes.c_void_p()
    _check(load().steps_cyl_resume(ctypes.byref(ctx), os.fsencode(path), int(device), ctypes.c_void_p(stream or None)))
    return ctx


class StepLog:
    """Per-step metrics as JSON lines appended to a file. Each line holds:
    - step, t and a;
    - wall_ms_per_step, the host wall time of the chunk's KDK steps and the
      diagnostics read-back, per step;
    - pair_images_per_s of the last force evaluation's pair kernel;
    - P (sum m p), L_z, the kinetic energy and the total mass, as
      steps_cyl_diagnostics returns them."""

    def __init__(self, path: str):
        self.path = path
        self.fh = open(path, "a")

    def write(self, step: int, diag, timing, wall_ms: float) -> dict:
        images, pair_ms = timing
        rec = {"step": int(step), "t": float(diag[6]), "a": float(diag[5]), "wall_ms_per_step": float(wall_ms),
               "pair_images_per_s": float(images / (pair_ms * 1e-3)) if pair_ms > 0 else None,
               "P": [float(x) for x in diag[0:3]], "L_z": float(diag[3]), "kinetic": float(diag[4]),
               "mass": float(diag[7])}
        self.fh.write(json.dumps(rec) + "\n")
        self.fh.flush()
        return rec

    def close(self):
        if self.fh:
            self.fh.close()
            self.fh = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Simulation:
    """Convenience owner of one context (numpy/torch arrays in, numpy out)."""

    def __init__(self, cfg: Config, pos, vel, m, h):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        vel = np.ascontiguousarray(vel, dtype=np.float64)
        self.n = pos.shape[0]
        cols = [np.ascontiguousarray(pos[:, k]) for k in range(3)] + [np.ascontiguousarray(vel[:, k]) for k in range(3)]
        self.cfg = cfg
        self.ctx = steps_cyl_init(cfg, self.n, *cols, np.ascontiguousarray(m, dtype=np.float64),
                                  np.ascontiguousarray(h, dtype=np.float64))

    def forces(self) -> np.ndarray:
        out = [np.zeros(self.n) for _ in range(3)]
        steps_cyl_forces(self.ctx, *out)
        return np.stack(out, 1)

    def forces_subset(self, idx) -> np.ndarray:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = [np.zeros(idx.shape[0]) for _ in range(3)]
        steps_cyl_forces_subset(self.ctx, idx, *out)
        return np.stack(out, 1)

    def step(self, dt: float, nsteps: int = 1):
        steps_cyl_kdk_step(self.ctx, dt, nsteps)

    def run(self, dt: float, nsteps: int, log: str | None = None, every: int = 1):
        """nsteps KDK steps of dt. With a log path, the steps run in chunks of
        `every` and one JSON line per chunk is appended to the file (StepLog)."""
        if log is None:
            return self.step(dt, nsteps)
        if every < 1:
            raise ValueError("every must be >= 1")
        with StepLog(log) as lg:
            done = 0
            while done < nsteps:
                k = min(every, nsteps - done)
                t0 = time.perf_counter()
                self.step(dt, k)
                diag = self.diagnostics()  # reads back to the host: the chunk has finished
                wall_ms = (time.perf_counter() - t0) * 1e3 / k
                done += k
                lg.write(done, diag, self.last_timing(), wall_ms)

    def state(self):
        out = [np.zeros(self.n) for _ in range(6)]
        a, t = steps_cyl_get_state(self.ctx, *out)
        return np.stack(out[:3], 1), np.stack(out[3:], 1), a, t

    def set_precision(self, precision: int):
        steps_cyl_set_precision(self.ctx, precision)

    def diagnostics(self) -> np.ndarray:
        return steps_cyl_diagnostics(self.ctx)

    def last_timing(self):
        return steps_cyl_last_timing(self.ctx)

    def checkpoint(self, path: str):
        steps_cyl_checkpoint(self.ctx, path)

    @classmethod
    def resume(cls, path: str, device: int = 0, stream: int = 0):
        """A Simulation continuing from a checkpoint file."""
        sim = cls.__new__(cls)
        sim.n = _ckpt_n(path)
        sim.cfg = None
        sim.ctx = steps_cyl_resume(path, device, stream)
        return sim

    def close(self):
        if self.ctx:
            steps_cyl_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
