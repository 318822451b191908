"""Builds libjpsi.so (sm_103a) in-tree with nvcc, and libjpsi_checked.so, the
same library with bounds-checked stores (-DJPSI_CHECKED=1) that the tests run
the parity suite on: every translation unit compiled in parallel, statically
linked CUDA runtime."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libjpsi.so")
LIB_CHECKED = os.path.join(HERE, "libjpsi_checked.so")
SOURCES = ["jpsi_kernels.cu", "jpsi_api.cu"]
# jpsi_kernels.cu once more with the time tests of free-streaming windows
STREAM_UNIT = ("jpsi_kernels.cu", "jpsi_kernels_stream.o", ["-DJPSI_STREAM=1"])
# the kernels again with bounds-checked stores (the host code is shared)
CHECKED_UNITS = [("jpsi_kernels.cu", "jpsi_kernels_checked.o", ["-DJPSI_CHECKED=1"]),
                 ("jpsi_kernels.cu", "jpsi_kernels_stream_checked.o", ["-DJPSI_STREAM=1", "-DJPSI_CHECKED=1"])]
HEADERS = ["jpsi_device.cuh", "jpsi_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xptxas", "-v", "-Xcompiler", "-fPIC,-O2",
              "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB_CHECKED):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "jpsi.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(unit):
        src, obj_name, extra = unit
        obj = os.path.join(BUILD, obj_name)
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        with open(os.path.join(BUILD, obj_name.replace(".o", ".log")), "w") as f:
            f.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src} {extra}:\n{r.stderr[-6000:]}")
        return obj

    units = [(src, src.replace(".cu", ".o"), []) for src in SOURCES] + [STREAM_UNIT]
    with ThreadPoolExecutor(len(units) + len(CHECKED_UNITS)) as ex:
        objs = list(ex.map(compile_one, units + CHECKED_UNITS))
    api = objs[SOURCES.index("jpsi_api.cu")]
    plain_objs, checked_objs = objs[:len(units)], [api] + objs[len(units):]
    for lib, lib_objs in ((LIB, plain_objs), (LIB_CHECKED, checked_objs)):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *lib_objs, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, lib)
    if verbose:
        for src in SOURCES:
            print(open(os.path.join(BUILD, src.replace(".cu", ".log"))).read())
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
