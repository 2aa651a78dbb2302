"""In-tree build of the CUDA library ``libsteps_cyl.so`` for sm_103a.

``build()`` runs nvcc once per changed source (a stamp of the source contents
and flags sits next to the library) and returns the library path.
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libsteps_cyl.so")
# the index-checked variant (every computed index of the symmetric kernels
# checked against its buffer): a test build, loaded when STEPS_CYL_INDEX_CHECKED=1
LIB_CHECKED = os.path.join(PKG, "libsteps_cyl_checked.so")
CHECKED_DEFS = ["-DSTEPS_DEBUG_INDEX=1"]
SOURCES = ["steps_cyl.cu", "steps_cyl_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared"]
_lock = threading.Lock()


def _nvcc() -> str:
    env = os.environ.get("NVCC")
    if env:
        return env
    if os.path.exists("/usr/local/cuda/bin/nvcc"):
        return "/usr/local/cuda/bin/nvcc"
    return "nvcc"


def _digest(extra=()) -> str:
    h = hashlib.sha256()
    files = sorted(os.listdir(CSRC)) + ["../../include/steps_cyl.h"]
    for f in files:
        path = os.path.normpath(os.path.join(CSRC, f))
        if os.path.isfile(path):
            h.update(f.encode())
            with open(path, "rb") as fh:
                h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS + list(extra)).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build the library (checked: the index-checked test variant) unless its
    stamp matches the sources; returns its path."""
    lib, extra = (LIB_CHECKED, CHECKED_DEFS) if checked else (LIB, [])
    with _lock:
        stamp = lib + ".stamp"
        dig = _digest(extra)
        if not force and os.path.exists(lib) and os.path.exists(stamp):
            with open(stamp) as fh:
                if fh.read().strip() == dig:
                    return lib
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [_nvcc(), *ARCH, *FLAGS, *extra, "-I" + INCLUDE, "-o", tmp] + [os.path.join(CSRC, s) for s in SOURCES]
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
        with open(stamp, "w") as fh:
            fh.write(dig)
        return lib


if __name__ == "__main__":
    print(build(verbose=True))
