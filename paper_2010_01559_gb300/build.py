"""Build librbe.so (the CUDA library behind include/rbe.h) in-tree for sm_103a.

Each .cu file under csrc/ is compiled in parallel with nvcc into an object, and
the objects are linked into ``_build/librbe.so`` next to this file.  Host code
is compiled without floating-point contraction so that the FP64 sampling
table is reproducible bit for bit.

``build(check_bounds=True)`` makes the bounds-checked variant
``_build/checked/librbe.so`` (compiled with -DRBE_CHECK_BOUNDS): every index the
kernels compute from data (cell ids, sorted slots, neighbour-list entries,
caller indices) is tested against its array before the access; a failed test
skips the access and latches RBE_ERR_BOUNDS, reported by the next rbe_sync.
It is a debugging aid for the tests, not the product's library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librbe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -ftz=true: FP32 subnormals flush to zero, so the approximate reciprocal,
# square root and exponential of the pair terms need no subnormal fix-ups (no
# FP32 quantity of the method comes near 1e-38; FP64 work is unaffected).
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-ftz=true", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-Wno-deprecated-declarations",
              "-diag-suppress", "1444", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librbe")
    return exe


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "rbe.h"),
                                                                  os.path.abspath(__file__)]


CHECKED_LIB = os.path.join(BUILD, "checked", "librbe.so")


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          check_bounds: bool = False) -> str:
    lib = CHECKED_LIB if check_bounds else LIB
    if not force and up_to_date(lib):
        return lib
    out_dir = os.path.dirname(lib)
    os.makedirs(out_dir, exist_ok=True)
    exe = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    if check_bounds:
        extra += ["-DRBE_CHECK_BOUNDS"]

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [exe] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(compile_one, _sources()))
    if verbose or ptxas_info:
        for _, log in results:
            if log:
                print(log)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
