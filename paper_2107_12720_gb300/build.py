"""Builds libtrim.so (the CUDA library behind include/trim.h) in-tree for sm_103a.

    python -m paper_2107_12720_gb300.build [--force]

Each .cu file is compiled in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo), then linked with a
static CUDA runtime into paper_2107_12720_gb300/libtrim.so.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtrim.so")
# (source, extra nvcc flags, object): the persistent kernel is built once per
# flavour (variant set), see TRIM_MODES in trim_kernels.cu
UNITS = [("trim_kernels.cu", ["-DTRIM_MODES=1"], "trim_kernels_m1.o"),
         ("trim_kernels.cu", ["-DTRIM_MODES=2"], "trim_kernels_m2.o"),
         ("trim_kernels.cu", ["-DTRIM_MODES=4"], "trim_kernels_m4.o"),
         ("trim_kernels.cu", ["-DTRIM_MODES=9"], "trim_kernels_m9.o"),
         ("trim_kernels.cu", ["-DTRIM_MODES=10"], "trim_kernels_m10.o"),
         ("trim_kernels.cu", ["-DTRIM_MODES=12"], "trim_kernels_m12.o"),
         ("trim_kernels.cu", ["-DTRIM_MODES=15"], "trim_kernels_m15.o"),
         ("trim_kernels.cu", ["-DTRIM_MODES=17"], "trim_kernels_m17.o"),
         ("trim_kernels.cu", ["-DTRIM_MODES=34"], "trim_kernels_m34.o"),
         ("trim_kernels.cu", ["-DTRIM_MODES=36"], "trim_kernels_m36.o"),
         ("trim_aux.cu", [], "trim_aux.o"),
         ("trim_scc.cu", [], "trim_scc.o"),
         ("trim_api.cu", [], "trim_api.o"),
         ("trim_noalloc.cu", [], "trim_noalloc.o"),
         ("mlp.cu", [], "mlp.o")]
SOURCES = sorted({u[0] for u in UNITS})
HEADERS = ["trim_internal.cuh", os.path.join("..", "..", "include", "trim.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in HEADERS]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    for src, extra, o in UNITS:
        obj = os.path.join(BUILD, o)
        objs.append(obj)
        cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + out.decode(errors="replace"))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
