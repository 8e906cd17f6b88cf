"""In-tree build of liblc.so for sm_103a (nvcc, one -gencode, parallel TUs).

build(debug=True) makes the checked build, liblc_debug.so (-DLC_DEBUG=1:
index checks in the kernels, see include/lc.h); the binding loads it instead
of liblc.so when the environment sets LC_DEBUG=1."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liblc.so")
LIB_DEBUG = os.path.join(LIBDIR, "liblc_debug.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "--extended-lambda", "-lineinfo", "-Xcompiler", "-fPIC",
          "-Xcompiler", "-fvisibility=hidden"]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(HERE, "..", "include", "lc.h")]


def debug_requested() -> bool:
    return os.environ.get("LC_DEBUG", "0") not in ("", "0")


def lib_path(debug: bool | None = None) -> str:
    return LIB_DEBUG if (debug_requested() if debug is None else debug) else LIB


def up_to_date(debug: bool | None = None) -> bool:
    lib = lib_path(debug)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = lib_path(debug)
    if not force and up_to_date(debug):
        return lib
    objdir = os.path.join(LIBDIR, "debug") if debug else LIBDIR
    os.makedirs(objdir, exist_ok=True)
    objs = []
    flags = CFLAGS + (["-DLC_DEBUG=1"] if debug else [])

    def compile_one(src: str) -> str:
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [NVCC, *ARCH, *flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = f"{lib}.{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fvisibility=hidden"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
