"""Build libhmi.so (the CUDA path) in-tree with nvcc for sm_103a.

Each .cu file is compiled in parallel to an object, then linked into
``paper_1907_04393_gb300/_lib/libhmi.so``.  No CMake, no PyTorch extension
machinery: the library is a plain C-ABI shared object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libhmi.so")
# the debug build: compiled with HMI_DEBUG, so that every computed index of the
# per-pixel kernels is bounds-checked (a failed check records an error flag and
# skips the access)
LIB_DEBUG = os.path.join(OUT_DIR, "libhmi_debug.so")
SOURCES = ["hmi_frame.cu", "hmi_tick.cu", "hmi_cc.cu", "hmi_learn.cu", "hmi_mix.cu", "hmi_api.cu", "hmi_tune.cu", "hmi_server.cu",
           "hmi_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhmi.so")


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    return files + [os.path.join(ROOT, "include", "hmi.h")]


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(debug):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    suffix = "_debug.o" if debug else ".o"

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT_DIR, src.replace(".cu", suffix))
        cmd = [cc, *ARCH, *NVCC_FLAGS, *(["-DHMI_DEBUG"] if debug else []), *inc, "-c",
               os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
