"""Refusals that the C ABI makes on the host, before its first CUDA call, so
these run without a GPU.

- Checkpoints: steps_cyl_resume refuses corrupt files. The files are written
  here from a ctypes mirror of the library's checkpoint header. A layout
  mismatch would show up as "not a checkpoint" in place of the specific refusal.
- Parameters: steps_cyl_init and steps_cyl_tail_sums refuse window and
  near-range settings outside their domain (eq. ForceCylindrical's window, and
  the infinite window of Sect. 2.2, whose tail sums the images to |k| = 512 one
  by one)."""
import ctypes
import math

import numpy as np
import pytest

from paper_2602_20787_gb300 import steps_cyl as sc

d, i32 = ctypes.c_double, ctypes.c_int32


class CkptHeader(ctypes.Structure):
    _fields_ = [
        ("magic", ctypes.c_char * 8), ("version", ctypes.c_uint32), ("header_bytes", ctypes.c_uint32),
        ("p", sc.Params), ("n", ctypes.c_int64),
        ("a", d), ("t", d), ("rho0", d), ("bg_dr", d), ("bound_med", d), ("bound_p999", d),
        ("steps_since_order", i32), ("steps_since_check", i32), ("surr_ok", i32), ("bgK", i32),
        ("surr", ctypes.c_float * sc.STEPS_SURR_NPARAM),
        ("tab_ok", i32), ("tab_nx", i32), ("tab_ny", i32), ("pad", i32),
        ("tab_dR_max", d), ("tab_bound_med", d), ("tab_bound_p999", d),
        ("tree_evals", ctypes.c_uint64), ("tree_fixed", i32), ("rad_nb", i32),
        ("tree_frame", d * 9), ("rad_rmax", d),
    ]


N = 4


def write_ckpt(path, *, perm=None, bgK=8, bg_dr=0.1, a=1.0, t=0.0, rho0=0.1, n=N, version=4, extra=b"",
               cut=0, background=sc.STEPS_BG_FINITE):
    hd = CkptHeader()
    hd.magic = b"STEPSCYL"
    hd.version = version
    hd.header_bytes = ctypes.sizeof(CkptHeader)
    hd.p = sc.steps_cyl_params_default()
    hd.p.background = background
    hd.p.stream = None
    hd.n = n
    hd.a, hd.t, hd.rho0, hd.bg_dr = a, t, rho0, bg_dr
    hd.bgK = bgK
    body = bytes(hd)
    if bgK:
        body += np.zeros(bgK + 4).tobytes()
    arr = np.zeros((11, N))
    arr[0] = [0.1, 0.2, 0.3, 0.4]
    arr[2] = [0.1, 0.3, 0.5, 0.7]
    arr[6:8] = 1.0
    body += arr.tobytes()
    body += np.asarray(np.arange(N) if perm is None else perm, dtype=np.int32).tobytes()
    body += extra
    if cut:
        body = body[:-cut]
    with open(path, "wb") as fh:
        fh.write(body)
    return path


@pytest.fixture(scope="module")
def lib():
    from paper_2602_20787_gb300 import build
    build.build()
    return sc.load(build_if_missing=False)


def refused(path, what):
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_resume(str(path))
    assert e.value.code == sc.STEPS_EINVAL
    assert what in str(e.value), str(e.value)


def test_mirror_matches_the_binding_offset(lib):
    # the binding reads n at the offset that follows magic, version, size and the parameters
    assert CkptHeader.n.offset == 8 + 4 + 4 + ctypes.sizeof(sc.Params)


@pytest.mark.parametrize("perm", [[0, 1, 1, 3], [0, 1, 2, 7], [0, 1, 2, -1], [3, 3, 3, 3]])
def test_permutation_must_be_one_of_0_to_n(lib, tmp_path, perm):
    refused(write_ckpt(tmp_path / "c", perm=perm), "permutation")


@pytest.mark.parametrize("kw", [dict(bgK=0), dict(bg_dr=0.0), dict(bg_dr=math.nan), dict(bg_dr=math.inf)])
def test_finite_background_needs_its_table(lib, tmp_path, kw):
    refused(write_ckpt(tmp_path / "c", **kw), "background table")


@pytest.mark.parametrize("kw", [dict(a=0.0), dict(a=-1.0), dict(a=math.nan), dict(t=math.inf), dict(rho0=-1.0),
                                dict(rho0=math.nan)])
def test_scale_factor_time_and_density(lib, tmp_path, kw):
    refused(write_ckpt(tmp_path / "c", **kw), "a, t or rho0")


@pytest.mark.parametrize("kw", [dict(cut=4), dict(cut=100), dict(extra=b"\0"), dict(n=1 << 30), dict(n=3)])
def test_size_must_match_the_header(lib, tmp_path, kw):
    refused(write_ckpt(tmp_path / "c", **kw), "truncated or has trailing bytes")


@pytest.mark.parametrize("kw", [dict(version=3), dict(n=1), dict(bgK=-2)])
def test_foreign_headers(lib, tmp_path, kw):
    refused(write_ckpt(tmp_path / "c", **kw), "not a checkpoint")


def test_a_background_table_is_optional_without_the_finite_background(lib, tmp_path):
    # the same file without a table passes every host check when the background
    # does not need one; the call then reaches the device (not made here), so
    # only the refusals above are asserted, and this file is checked to be well formed
    path = write_ckpt(tmp_path / "c", bgK=0, background=sc.STEPS_BG_OFF)
    size = ctypes.sizeof(CkptHeader) + N * (11 * 8 + 4)
    assert path.stat().st_size == size


def init_refused(cfg, what, n=4):
    d = np.zeros(n)
    arrs = [np.linspace(0.1, 0.4, n), np.zeros(n), np.linspace(0.1, 0.7, n), d, d, d, np.ones(n), np.ones(n)]
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_init(cfg, n, *arrs)
    assert e.value.code == sc.STEPS_EINVAL
    assert what in str(e.value), str(e.value)


@pytest.mark.parametrize("n0", [-1, 512, 4000])
def test_infinite_window_near_range(lib, n0):
    cfg = sc.Config(n_cut=0, n0=n0, tail=sc.STEPS_TAIL_TABLE, background=sc.STEPS_BG_INFINITE)
    init_refused(cfg, "n0 must be in [0, 512)")


def test_nearest_image_table_only(lib):
    # n0 = 0 (the table over the nearest image alone) is for the table tail only
    cfg = sc.Config(n_cut=0, n0=0, tail=sc.STEPS_TAIL_SURROGATE, background=sc.STEPS_BG_INFINITE)
    init_refused(cfg, "needs STEPS_TAIL_TABLE")
    init_refused(sc.Config(n_cut=8, n0=0, tail=sc.STEPS_TAIL_SURROGATE), "learned tail needs n0 in [1, n_cut)")
    init_refused(sc.Config(n_cut=8, n0=-1), "n0 must be >= 0")


@pytest.mark.parametrize("kw,what", [(dict(n_cut=4097), "n_cut must be in"), (dict(n_cut=-1), "n_cut must be in"),
                                     (dict(n_cut=8, n0=8, tail=sc.STEPS_TAIL_TABLE), "table tail needs n0 in [0, n_cut)"),
                                     (dict(theta=0.5, force=sc.STEPS_FORCE_OCTREE), "octree needs the infinite"),
                                     (dict(topology=sc.STEPS_TOPO_R3, background=sc.STEPS_BG_FINITE), "R^3 topology")])
def test_init_parameters(lib, kw, what):
    init_refused(sc.Config(**kw), what)


def test_init_particle_count(lib):
    init_refused(sc.Config(), "n must be in", n=1)


@pytest.mark.parametrize("n_cut,n0", [(4097, 4), (-1, 0), (8, 8), (8, -1), (0, 512), (0, 1000)])
def test_tail_sums_domain(lib, n_cut, n0):
    smp = np.array([[0.5, 0.1, 0.01]])
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_tail_sums(smp, n_cut, n0)
    assert e.value.code == sc.STEPS_EINVAL


def test_binding_checks_dtype_and_layout(lib):
    n = 4
    good = [np.linspace(0.1, 0.4, n), np.zeros(n), np.linspace(0.1, 0.7, n)] + [np.zeros(n)] * 3 + [np.ones(n)] * 2
    bad_dtype = list(good)
    bad_dtype[6] = np.ones(n, dtype=np.float32)
    with pytest.raises(TypeError):
        sc.steps_cyl_init(sc.Config(), n, *bad_dtype)
    strided = list(good)
    strided[0] = np.linspace(0.1, 0.8, 2 * n)[::2]
    with pytest.raises(ValueError):
        sc.steps_cyl_init(sc.Config(), n, *strided)
    with pytest.raises(TypeError):
        sc._ptr([1.0, 2.0])
    assert sc._ptr(None) is None


def test_noalloc_binding_refuses_host_arrays_before_the_library():
    # the allocation-free entry point takes device memory only; the binding
    # refuses numpy arrays (host memory) before it calls the library
    pytest.importorskip("torch")
    x = np.zeros(16)
    with pytest.raises(sc.StepsError) as e:
        sc.steps_cyl_pair_accel_noalloc(x, x, x, x, x, 1.0, 1.0, 4, sc.STEPS_FP32_KAHAN, x, x, x)
    assert e.value.code == sc.STEPS_EINVAL
