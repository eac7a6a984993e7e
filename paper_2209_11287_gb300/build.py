"""Build libsj (the CUDA library behind include/simjoin.h) for sm_103a.

Each .cu under csrc/ is compiled by nvcc in parallel and linked into
``_build/libsj.so`` in this package directory (in-tree, ignored by git).  The
CUDA runtime is linked statically, so the library loads on a machine without a
GPU driver (calls then fail with SJ_ERR_CUDA).
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsj.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "simjoin.h")]


# The bounds-checking variant (tile kernels check every candidate, query and
# stage index and report the first failing site instead of touching memory):
# a second library, built on request for its test.
DEBUG_BUILD = os.path.join(BUILD, "debug_bounds")
DEBUG_LIB = os.path.join(DEBUG_BUILD, "libsj.so")


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    lib = DEBUG_LIB if debug_bounds else LIB
    out_dir = DEBUG_BUILD if debug_bounds else BUILD
    extra = ["-DSJ_DEBUG_BOUNDS"] if debug_bounds else []
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    srcs = _sources()

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=min(16, len(srcs), max(4, os.cpu_count() or 4))) as ex:
        res = list(ex.map(compile_one, srcs))
    if verbose:
        for _, err in res:
            sys.stderr.write(err)
    objs = [o for o, _ in res]
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))


def build_peaks() -> str:
    """Build the arithmetic-throughput micro-benchmark (peaks/sj_peaks.cu) as
    the executable _build/sj_peaks."""
    os.makedirs(BUILD, exist_ok=True)
    src = os.path.join(HERE, "peaks", "sj_peaks.cu")
    exe = os.path.join(BUILD, "sj_peaks")
    if os.path.exists(exe) and os.path.getmtime(exe) >= os.path.getmtime(src):
        return exe
    subprocess.run([_nvcc(), *ARCH, "-O3", "-std=c++17", "-o", exe, src], check=True)
    return exe
