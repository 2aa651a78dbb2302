"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/*.h declares (no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

from tests.conftest import ROOT


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mth in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(steps_cyl_\w+)\s*\(", text, flags=re.M):
            names.add(mth.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2602_20787_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("steps_cyl_init", "steps_cyl_forces", "steps_cyl_kdk_step", "steps_cyl_free"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_symbol():
    from paper_2602_20787_gb300 import steps_cyl
    assert set(declared_functions()) <= set(steps_cyl._EXPORTS)


def test_host_only_entry_points(lib):
    from paper_2602_20787_gb300 import steps_cyl as sc
    p = sc.steps_cyl_params_default()
    assert p.n_cut == 16 and p.precision == sc.STEPS_FP32_KAHAN and p.G == 1.0
    lib.steps_cyl_strerror.restype = ctypes.c_char_p
    assert lib.steps_cyl_strerror(sc.STEPS_EINVAL) == b"invalid argument"
    assert lib.steps_cyl_strerror(12345) == b"unknown status"


def test_library_is_sm103a():
    from paper_2602_20787_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2602_20787_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(path).read()
            assert "import oracle" not in src and "from oracle" not in src and "steps_oracle" not in src, path


def test_binding_constants_match_the_header():
    from paper_2602_20787_gb300 import steps_cyl
    text = open(os.path.join(ROOT, "include", "steps_cyl.h")).read()
    defs = dict(re.findall(r"^#define (STEPS_\w+) (-?\d+)\b", text, flags=re.M))
    shared = [k for k in defs if hasattr(steps_cyl, k)]
    assert "STEPS_TABLE_READ_TSC" in shared and len(shared) > 10
    for k in shared:
        assert getattr(steps_cyl, k) == int(defs[k]), k


def test_table_read_refuses_without_a_context(lib):
    from paper_2602_20787_gb300 import steps_cyl as sc
    lib.steps_cyl_set_table_read.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    assert lib.steps_cyl_set_table_read(None, sc.STEPS_TABLE_READ_TSC) == sc.STEPS_EINVAL
