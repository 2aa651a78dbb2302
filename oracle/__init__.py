"""FP64 CPU oracle for the S1xR2 StePS hot path (arXiv 2602.20787).

TEST INFRASTRUCTURE ONLY. The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The product path (the
CUDA library and its binding) never imports this package, and this package
never imports the product: the two share no code. The only module both sides
read is the seeded input generator ``paper_2602_20787_gb300.ics``, which holds
no force, integrator or surrogate arithmetic.

The C source ``steps_oracle.c`` is compiled with gcc into ``liboracle.so`` next
to it (``build()``); this module wraps it with ctypes and adds numpy-facing
helpers. Each wrapper names the equation of the paper it evaluates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "steps_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MLP_HIDDEN = 32
MLP_NW = MLP_HIDDEN * 3 + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + 2 * MLP_HIDDEN + 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP). Returns the library path."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "steps_oracle.h")))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC,
                   "-lm"]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, _LIB)
    return _LIB


class Cosmo(ctypes.Structure):
    """Eqs. Friedmann / DEdensity / CPLw0wa parameters; comoving=0 is static space."""
    _fields_ = [("H0", ctypes.c_double), ("Omega_m", ctypes.c_double), ("Omega_r", ctypes.c_double),
                ("Omega_L", ctypes.c_double), ("w0", ctypes.c_double), ("wa", ctypes.c_double),
                ("comoving", ctypes.c_int32)]


class SurrCfg(ctypes.Structure):
    """Surrogate definition constants (this project's; see or_tail_surrogate)."""
    _fields_ = [("n_cut", ctypes.c_int32), ("n0", ctypes.c_int32), ("dR_max", ctypes.c_double),
                ("out_mu", ctypes.c_double * 2), ("out_sc", ctypes.c_double * 2)]


def make_surr_cfg(n_cut, n0, dR_max, out_mu=(0.0, 0.0), out_sc=(1.0, 1.0)):
    c = SurrCfg()
    c.n_cut, c.n0, c.dR_max = int(n_cut), int(n0), float(dR_max)
    c.out_mu[0], c.out_mu[1] = out_mu
    c.out_sc[0], c.out_sc[1] = out_sc
    return c


TABLE_CIC, TABLE_TSC = 0, 1


class TableCfg(ctypes.Structure):
    _fields_ = [("n_cut", ctypes.c_int32), ("n0", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("dR_max", ctypes.c_double), ("read", ctypes.c_int32), ("pad", ctypes.c_int32)]


def make_table_cfg(n_cut, n0, nx, ny, dR_max, read=TABLE_CIC):
    """Table definition; read = TABLE_CIC (bilinear) or TABLE_TSC (Sect. 2.3)."""
    c = TableCfg()
    c.n_cut, c.n0, c.nx, c.ny, c.dR_max = int(n_cut), int(n0), int(nx), int(ny), float(dR_max)
    c.read = int(read)
    return c


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i32, i64, p = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        L.or_spline_F.argtypes = [d, d]; L.or_spline_F.restype = d
        L.or_spline_F_over_r.argtypes = [d, d]; L.or_spline_F_over_r.restype = d
        L.or_image_force.argtypes = [d, d, d, d, d, i32, p]; L.or_image_force.restype = ctypes.c_int
        L.or_pair_field.argtypes = [i64, p, p, p, p, p, d, d, i32, i64, p, p, p, p]
        L.or_pair_field.restype = None
        L.or_cylinder_field.argtypes = [d, d, d, d, d]; L.or_cylinder_field.restype = d
        L.or_background_field.argtypes = [i64, p, p, d, d, d, d, p, p]
        L.or_background_field.restype = None
        L.or_hubble.argtypes = [ctypes.POINTER(Cosmo), d]; L.or_hubble.restype = d
        L.or_a_of_t_step.argtypes = [ctypes.POINTER(Cosmo), d, d]; L.or_a_of_t_step.restype = d
        L.or_kdk_factors.argtypes = [ctypes.POINTER(Cosmo), d, d, p, p, p, p]
        L.or_kdk_factors.restype = None
        L.or_kdk.argtypes = [i64, p, p, p, p, p, p, p, p, d, d, i32, d, d, i32,
                             ctypes.POINTER(Cosmo), p, p, d, i32]
        L.or_kdk_topo.argtypes = [i64, p, p, p, p, p, p, p, p, d, d, i32, d, d, i32, i32,
                                  ctypes.POINTER(Cosmo), p, p, d, i32]
        L.or_kdk_topo.restype = ctypes.c_int
        L.or_pair_field_r3.argtypes = [i64, p, p, p, p, p, d, i64, p, p, p, p]; L.or_pair_field_r3.restype = None
        L.or_background_sphere.argtypes = [i64, p, p, p, d, d, p, p, p]; L.or_background_sphere.restype = None
        L.or_kdk.restype = ctypes.c_int
        L.or_tree_field.argtypes = [i64, p, p, p, p, p, d, d, d, i32, p, p, d, i32, d, d, i64, p, p, p, p, p]
        L.or_tree_field.restype = ctypes.c_int
        L.or_tree_field_r3.argtypes = [i64, p, p, p, p, p, d, d, d, i32, p, p, d, i64, p, p, p, p, p]
        L.or_tree_field_r3.restype = ctypes.c_int
        L.or_tree_order.argtypes = [i64, p, p, p, d, d, d, d, p, p]
        L.or_tree_order.restype = ctypes.c_int
        L.or_tail_sums.argtypes = [d, d, d, d, i32, i32, p, p]; L.or_tail_sums.restype = None
        L.or_diagnostics.argtypes = [i64, p, p, p, p, p, p, d, p]; L.or_diagnostics.restype = None
        L.or_mlp_forward.argtypes = [p, p, p]; L.or_mlp_forward.restype = None
        L.or_mlp_loss_grad.argtypes = [p, i64, p, p, p]; L.or_mlp_loss_grad.restype = d
        L.or_adam_step.argtypes = [i64, p, p, p, p, d, d, d, d, i64]; L.or_adam_step.restype = None
        L.or_num_threads.argtypes = []; L.or_num_threads.restype = i32
        L.or_tail_base.argtypes = [d, d, i32, i32, p, p]; L.or_tail_base.restype = None
        L.or_tail_envelope.argtypes = [d, d, i32, p, p]; L.or_tail_envelope.restype = None
        L.or_surrogate_inputs.argtypes = [d, d, d, i32, d, p]; L.or_surrogate_inputs.restype = None
        L.or_tail_surrogate.argtypes = [d, d, d, p, ctypes.POINTER(SurrCfg), p, p]
        L.or_tail_surrogate.restype = None
        L.or_pair_field_surrogate.argtypes = [i64, p, p, p, p, p, d, d, p, ctypes.POINTER(SurrCfg), i64, p, p, p, p]
        L.or_pair_field_surrogate.restype = None
        L.or_image_sums_inf.argtypes = [d, d, d, i32, p, p]; L.or_image_sums_inf.restype = None
        L.or_pair_field_inf.argtypes = [i64, p, p, p, p, p, d, d, i64, p, p, p, p]; L.or_pair_field_inf.restype = None
        L.or_tail_base_inf.argtypes = [d, d, i32, p, p]; L.or_tail_base_inf.restype = None
        L.or_ewald_tail.argtypes = [d, d, i32, d, i32, i32, p, p]; L.or_ewald_tail.restype = None
        T = ctypes.POINTER(TableCfg)
        L.or_tail_residual.argtypes = [d, d, i32, i32, p]; L.or_tail_residual.restype = None
        L.or_tail_table_build.argtypes = [T, p]; L.or_tail_table_build.restype = None
        L.or_tail_table_read.argtypes = [p, T, d, d, p]; L.or_tail_table_read.restype = None
        L.or_tail_table.argtypes = [d, d, d, p, T, p, p]; L.or_tail_table.restype = None
        L.or_pair_field_table.argtypes = [i64, p, p, p, p, p, d, d, p, T, i64, p, p, p, p]
        L.or_pair_field_table.restype = None
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().or_num_threads())


def spline_F(r: float, h: float) -> float:
    """Eq. Force_spline_kernel."""
    return lib().or_spline_F(float(r), float(h))


def spline_F_over_r(r: float, h: float) -> float:
    """Eq. Force_spline_kernel divided by r (finite at r = 0)."""
    return lib().or_spline_F_over_r(float(r), float(h))


def image_force(r, h: float, L: float, n_cut: int):
    """Eq. ForceCylindrical per unit G. Returns (force[3], images used)."""
    out = np.zeros(3)
    cnt = lib().or_image_force(float(r[0]), float(r[1]), float(r[2]), float(h), float(L), int(n_cut),
                               _ptr(out))
    return out, cnt


def pair_field(pos, m, h, G: float, L: float, n_cut: int, idx=None):
    """Pair term of eq. ComovingEquationsOfMotionCylindrical times a^3 (no 1/a^3).

    pos: (N, 3) with z in [0, L). idx: optional subset of i. Returns (len(idx), 3).
    """
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    m = _f64(m); h = _f64(h)
    n = x.shape[0]
    if idx is None:
        ni, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ni, ip = idx.shape[0], _ptr(idx)
    gx, gy, gz = np.zeros(ni), np.zeros(ni), np.zeros(ni)
    lib().or_pair_field(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h), float(G), float(L), int(n_cut),
                        ni, ip, _ptr(gx), _ptr(gy), _ptr(gz))
    return np.stack([gx, gy, gz], axis=1)


def cylinder_field(varrho: float, R: float, Lw: float, G: float = 1.0, rho0: float = 1.0) -> float:
    """Eq. F_horiz (re-derived reading): radial mid-plane field of a finite cylinder."""
    return lib().or_cylinder_field(float(varrho), float(R), float(Lw), float(G), float(rho0))


def background_field(pos, R: float, Lw: float, G: float, rho0: float, mode: int = 1):
    """-F_h(rho) rho_hat (times a^3). mode 1: eq. F_horiz, 2: eq. F_horiz_infty, 0: off."""
    n = pos.shape[0]
    out = np.zeros((n, 3))
    if mode == 0:
        return out
    x, y = _f64(pos[:, 0]), _f64(pos[:, 1])
    if mode == 1:
        gx, gy = np.zeros(n), np.zeros(n)
        lib().or_background_field(n, _ptr(x), _ptr(y), float(R), float(Lw), float(G), float(rho0),
                                  _ptr(gx), _ptr(gy))
        out[:, 0], out[:, 1] = gx, gy
        return out
    rho = np.hypot(x, y)
    F = np.where(rho <= R, -2 * np.pi * G * rho0 * rho, -2 * np.pi * G * rho0 * R * R / np.maximum(rho, 1e-300))
    with np.errstate(invalid="ignore", divide="ignore"):
        out[:, 0] = np.where(rho > 0, -F * x / rho, 0.0)
        out[:, 1] = np.where(rho > 0, -F * y / rho, 0.0)
    return out


def make_cosmo(H0=1.0, Omega_m=0.3, Omega_L=0.7, Omega_r=0.0, w0=-1.0, wa=0.0, comoving=True):
    return Cosmo(float(H0), float(Omega_m), float(Omega_r), float(Omega_L), float(w0), float(wa),
                 1 if comoving else 0)


def hubble(c: Cosmo, a: float) -> float:
    """Eq. Friedmann: H(a)."""
    return lib().or_hubble(ctypes.byref(c), float(a))


def a_step(c: Cosmo, a: float, dt: float) -> float:
    """One RK4 step of da/dt = a H(a) (Sect. 2.3)."""
    return lib().or_a_of_t_step(ctypes.byref(c), float(a), float(dt))


def kdk_factors(c: Cosmo, a: float, dt: float):
    """(K1, D, K2, a_next): Int dt/a over each half step and Int dt/a^2 over the step."""
    out = np.zeros(4)
    lib().or_kdk_factors(ctypes.byref(c), float(a), float(dt), _ptr(out[0:]), _ptr(out[1:]),
                         _ptr(out[2:]), _ptr(out[3:]))
    return tuple(float(v) for v in out)


def kdk(pos, vel_p, m, h, G, L, n_cut, R_bg, rho0, background, c: Cosmo, a, t, dt, nsteps, topology=0):
    """KDK leapfrog (Sect. 2.1) on canonical momenta p = a^2 dx/dt. Returns (pos, p, a, t).
    topology 0: S1xR2 (z wrapped); 1: R^3 (background 0 or 3 = the radial sphere term)."""
    x, y, z = (_f64(pos[:, k]).copy() for k in range(3))
    px, py, pz = (_f64(vel_p[:, k]).copy() for k in range(3))
    m = _f64(m); h = _f64(h)
    a_ = ctypes.c_double(a); t_ = ctypes.c_double(t)
    rc = lib().or_kdk_topo(x.shape[0], _ptr(x), _ptr(y), _ptr(z), _ptr(px), _ptr(py), _ptr(pz), _ptr(m), _ptr(h),
                           float(G), float(L), int(n_cut), float(R_bg), float(rho0), int(background), int(topology),
                           ctypes.byref(c), ctypes.byref(a_), ctypes.byref(t_), float(dt), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle KDK allocation failed")
    return np.stack([x, y, z], 1), np.stack([px, py, pz], 1), a_.value, t_.value


def diagnostics(pos, p, m, a):
    """Sect. 1 conserved quantities of a state: (P[3] = sum m p, L_z = sum m (x p_y - y p_x),
    kinetic energy sum m |dx/dt|^2 / 2 with dx/dt = p / a^2, total mass). p: canonical momenta."""
    x, y = _f64(pos[:, 0]), _f64(pos[:, 1])
    px, py, pz = (_f64(p[:, k]) for k in range(3))
    m = _f64(m)
    out = np.zeros(6)
    lib().or_diagnostics(x.shape[0], _ptr(x), _ptr(y), _ptr(px), _ptr(py), _ptr(pz), _ptr(m), float(a), _ptr(out))
    return out


def tail_sums(dR, dzw, h, L, n_cut, n0):
    """Far-image tail (|k| > n0) of eq. ForceCylindrical in the wrapped frame: (SR, Sz)."""
    SR, Sz = ctypes.c_double(), ctypes.c_double()
    lib().or_tail_sums(float(dR), float(dzw), float(h), float(L), int(n_cut), int(n0),
                       ctypes.byref(SR), ctypes.byref(Sz))
    return SR.value, Sz.value


def mlp_forward(w, u):
    """3 -> 32 -> 32 -> 2 ReLU MLP in FP64. u: (3,) or (ns, 3)."""
    w = _f64(w)
    u = np.atleast_2d(_f64(u))
    y = np.zeros((u.shape[0], 2))
    for s in range(u.shape[0]):
        us = np.ascontiguousarray(u[s]); ys = np.zeros(2)
        lib().or_mlp_forward(_ptr(w), _ptr(us), _ptr(ys))
        y[s] = ys
    return y


def mlp_loss_grad(w, u, t):
    """Loss 1/(2ns) sum (y - t)^2 and its gradient by backpropagation (FP64)."""
    w = _f64(w); u = _f64(u); t = _f64(t)
    g = np.zeros(MLP_NW)
    loss = lib().or_mlp_loss_grad(_ptr(w), u.shape[0], _ptr(u), _ptr(t), _ptr(g))
    return loss, g


def adam_step(w, g, m1, m2, lr, beta1, beta2, eps, step):
    """In-place Adam update (FP64)."""
    lib().or_adam_step(w.shape[0], _ptr(w), _ptr(_f64(g)), _ptr(m1), _ptr(m2), float(lr), float(beta1),
                       float(beta2), float(eps), int(step))


def tail_base(dR, adz, n_cut, n0):
    """Order-1 Euler-Maclaurin continuum base of the far tail (units of L, |dz|)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().or_tail_base(float(dR), float(adz), int(n_cut), int(n0), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def tail_envelope(dR, adz, n0):
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().or_tail_envelope(float(dR), float(adz), int(n0), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def surrogate_inputs(dR, adz, h, n0, dR_max):
    u = np.zeros(3)
    lib().or_surrogate_inputs(float(dR), float(adz), float(h), int(n0), float(dR_max), _ptr(u))
    return u


def tail_surrogate(dR, dz, h, w, cfg):
    """Surrogate far tail (SR, SZ) in units of L for one pair."""
    w = _f64(w)
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().or_tail_surrogate(float(dR), float(dz), float(h), _ptr(w), ctypes.byref(cfg), ctypes.byref(a),
                            ctypes.byref(b))
    return a.value, b.value


def pair_field_surrogate(pos, m, h, G, L, w, cfg, idx=None):
    """Pair term with near images exact and the far tail from the surrogate."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    m = _f64(m); h = _f64(h); w = _f64(w)
    n = x.shape[0]
    if idx is None:
        ni, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ni, ip = idx.shape[0], _ptr(idx)
    gx, gy, gz = np.zeros(ni), np.zeros(ni), np.zeros(ni)
    lib().or_pair_field_surrogate(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h), float(G), float(L), _ptr(w),
                                  ctypes.byref(cfg), ni, ip, _ptr(gx), _ptr(gy), _ptr(gz))
    return np.stack([gx, gy, gz], axis=1)


def tail_residual(dR, adz, n_cut, n0):
    """Residual of the point-mass tail over the continuum base, in envelope units."""
    r = np.zeros(2)
    lib().or_tail_residual(float(dR), float(adz), int(n_cut), int(n0), _ptr(r))
    return r


def tail_table_build(cfg):
    """Correction table of the tail residual, shape (ny, nx, 2)."""
    tab = np.zeros((cfg.ny, cfg.nx, 2))
    lib().or_tail_table_build(ctypes.byref(cfg), _ptr(tab))
    return tab


def tail_table_read(tab, cfg, dR, adz):
    tab = _f64(tab)
    r = np.zeros(2)
    lib().or_tail_table_read(_ptr(tab), ctypes.byref(cfg), float(dR), float(adz), _ptr(r))
    return r


def tail_table(dR, dz, h, tab, cfg):
    """Table far tail (SR, SZ) in units of L for one pair."""
    tab = _f64(tab)
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().or_tail_table(float(dR), float(dz), float(h), _ptr(tab), ctypes.byref(cfg), ctypes.byref(a),
                        ctypes.byref(b))
    return a.value, b.value


def pair_field_table(pos, m, h, G, L, tab, cfg, idx=None):
    """Pair term with near images exact and the far tail from the correction table."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    m = _f64(m); h = _f64(h); tab = _f64(tab)
    n = x.shape[0]
    if idx is None:
        ni, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ni, ip = idx.shape[0], _ptr(idx)
    gx, gy, gz = np.zeros(ni), np.zeros(ni), np.zeros(ni)
    lib().or_pair_field_table(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h), float(G), float(L), _ptr(tab),
                              ctypes.byref(cfg), ni, ip, _ptr(gx), _ptr(gy), _ptr(gz))
    return np.stack([gx, gy, gz], axis=1)


def pair_field_r3(pos, m, h, G, idx=None):
    """R^3 pair field (eq. NewtonianForce, no images) per particle (or the listed ones)."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    m = _f64(m); h = _f64(h)
    n = x.shape[0]
    if idx is None:
        ni, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ni, ip = idx.shape[0], _ptr(idx)
    gx, gy, gz = np.zeros(ni), np.zeros(ni), np.zeros(ni)
    lib().or_pair_field_r3(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h), float(G), ni, ip, _ptr(gx), _ptr(gy),
                           _ptr(gz))
    return np.stack([gx, gy, gz], axis=1)


def background_sphere(pos, G, rho0):
    """The R^3 radial term +(4 pi G / 3) rho0 x."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    n = x.shape[0]
    gx, gy, gz = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().or_background_sphere(n, _ptr(x), _ptr(y), _ptr(z), float(G), float(rho0), _ptr(gx), _ptr(gy), _ptr(gz))
    return np.stack([gx, gy, gz], axis=1)


def image_sums_inf(dR, dzw, h, n0=-1):
    """Infinite-window image sums (SR, SZ) of the images |k| > n0 (all for n0 = -1)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().or_image_sums_inf(float(dR), float(dzw), float(h), int(n0), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def pair_field_inf(pos, m, h, G, L, idx=None):
    """Pair term with the infinite window (Ncut -> infinity)."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    m = _f64(m); h = _f64(h)
    n = x.shape[0]
    if idx is None:
        ni, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ni, ip = idx.shape[0], _ptr(idx)
    gx, gy, gz = np.zeros(ni), np.zeros(ni), np.zeros(ni)
    lib().or_pair_field_inf(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h), float(G), float(L), ni, ip, _ptr(gx),
                            _ptr(gy), _ptr(gz))
    return np.stack([gx, gy, gz], axis=1)


def ewald_tail(dR, dzw, n0, alpha, nmax, mmax):
    """Sect. 2.3 Ewald sums (SR, SZ) of the infinite line's images |k| > n0, units of L."""
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().or_ewald_tail(float(dR), float(dzw), int(n0), float(alpha), int(nmax), int(mmax), ctypes.byref(a),
                        ctypes.byref(b))
    return a.value, b.value


def tail_base_inf(dR, adz, n0):
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().or_tail_base_inf(float(dR), float(adz), int(n0), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def tree_field(pos, m, h, G, L, R_sim, n_cut, theta, leaf, zeta, phi, tab=None, tcfg=None, idx=None):
    """Octree field (Sect. 2.4) in the frame (zeta, phi) of every particle, or
    of the listed ones (idx): returns (g of shape (n or len(idx), 3), stats =
    nodes, leaves, depth, interactions of the groups walked). tab/tcfg: the
    correction-table form (near images plus table); None: the plain window of
    n_cut."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    m = _f64(m); h = _f64(h)
    n = x.shape[0]
    if idx is None:
        ni, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ni, ip = idx.shape[0], idx.ctypes.data_as(ctypes.c_void_p)
    gx, gy, gz = np.zeros(ni), np.zeros(ni), np.zeros(ni)
    stats = np.zeros(4, dtype=np.int64)
    tab_c = _f64(tab) if tab is not None else None
    tp = _ptr(tab_c) if tab_c is not None else None
    rc = lib().or_tree_field(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h), float(G), float(L), float(R_sim),
                             int(n_cut), tp, ctypes.byref(tcfg) if tcfg is not None else None, float(theta),
                             int(leaf), float(zeta), float(phi), ni, ip, _ptr(gx), _ptr(gy), _ptr(gz),
                             stats.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError(f"or_tree_field failed ({rc}): a particle outside the root cube" if rc == -1 else
                         f"or_tree_field failed ({rc})")
    return np.stack([gx, gy, gz], axis=1), stats


def tree_order(pos, L, R_sim, zeta, phi):
    """Keys and key order (ties by index) of the octree frame (zeta, phi)."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    n = x.shape[0]
    key = np.zeros(n, dtype=np.uint64)
    ordv = np.zeros(n, dtype=np.int64)
    rc = lib().or_tree_order(n, _ptr(x), _ptr(y), _ptr(z), float(L), float(R_sim), float(zeta), float(phi),
                             key.ctypes.data_as(ctypes.c_void_p), ordv.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError(f"or_tree_order failed ({rc})")
    return key, ordv


def tree_field_r3(pos, m, h, G, R_sim, theta, leaf, cen, axis, angle, idx=None):
    """The R^3 octree (Sect. 2.4) in the frame (domain centre cen, rotation by
    angle about the unit axis): (g, stats) as tree_field."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    m = _f64(m); h = _f64(h)
    n = x.shape[0]
    if idx is None:
        ni, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ni, ip = idx.shape[0], idx.ctypes.data_as(ctypes.c_void_p)
    gx, gy, gz = np.zeros(ni), np.zeros(ni), np.zeros(ni)
    stats = np.zeros(4, dtype=np.int64)
    c = _f64(cen); a = _f64(axis)
    rc = lib().or_tree_field_r3(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h), float(G), float(R_sim), float(theta),
                                int(leaf), _ptr(c), _ptr(a), float(angle), ni, ip, _ptr(gx), _ptr(gy), _ptr(gz),
                                stats.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError(f"or_tree_field_r3 failed ({rc})")
    return np.stack([gx, gy, gz], axis=1), stats
