"""Build the CUDA library in-tree: paper_2412_09775_gb300/lib/libwo_gb300.so.

Each translation unit under csrc/ is compiled by nvcc for sm_103a in
parallel, then linked into one shared library (static CUDA runtime, C ABI
from include/wo.h).  ``build(check=True)`` makes the WO_CHECK variant
(lib/libwo_gb300_check.so: every kernel tests the indices of its global
accesses and records the first out-of-range one instead of making it).
Run as ``python -m paper_2412_09775_gb300.build [--check]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libwo_gb300.so"
CHECK_LIB_NAME = "libwo_gb300_check.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-O3",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def lib_path(check: bool = False) -> str:
    return os.path.join(OUT_DIR, CHECK_LIB_NAME if check else LIB_NAME)


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _digest(check: bool = False) -> str:
    h = hashlib.sha256(b"check" if check else b"")
    for p in sorted(glob.glob(os.path.join(CSRC, "*")) + [os.path.join(INCLUDE, "wo.h")]):
        with open(p, "rb") as f:
            h.update(os.path.basename(p).encode())
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def _stamp(check: bool) -> str:
    return os.path.join(OUT_DIR, ".stamp_check" if check else ".stamp")


def up_to_date(check: bool = False) -> bool:
    stamp = _stamp(check)
    return os.path.exists(lib_path(check)) and os.path.exists(stamp) and open(stamp).read() == _digest(check)


def build(force: bool = False, verbose: bool = False, extra_flags=(), check: bool = False) -> str:
    """Compile every .cu under csrc/ and link the shared library; returns its path."""
    if not force and up_to_date(check):
        return lib_path(check)
    os.makedirs(OUT_DIR, exist_ok=True)
    bdir = BUILD_DIR + ("_check" if check else "")
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    srcs = _sources()
    defs = ["-DWO_CHECK=1"] if check else []

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *defs, *extra_flags, "-I", INCLUDE, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib_path(check) + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path(check))
    with open(_stamp(check), "w") as f:
        f.write(_digest(check))
    return lib_path(check)


if __name__ == "__main__":
    force = "--force" in sys.argv
    print(build(force=force, verbose="-v" in sys.argv, check="--check" in sys.argv))
