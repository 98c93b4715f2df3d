"""CPU oracle for graph trimming -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never imports, links or executes anything here.

The oracle is plain sequential C (``oracle.c``, compiled with gcc on first use)
plus a double-precision numpy reference of the scheduler MLP (``mlp_ref.py``).
Each function cites the passage of Guo & Sekerinski (arXiv 2107.12720) it
follows; see ``oracle.c`` for the definitions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

LIVE = 0xFFFFFFFF
MASKED = 0xFFFFFFFE

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (single-threaded, -O2) if stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
            u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
            lib.or_transpose.restype = ctypes.c_int
            lib.or_transpose.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u32p]
            lib.or_peel.restype = ctypes.c_uint32
            lib.or_peel.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u32p, u8p]
            lib.or_ac6.restype = ctypes.c_uint32
            lib.or_ac6.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u8p,
                                   ctypes.POINTER(ctypes.c_uint64)]
            lib.or_ac3.restype = ctypes.c_uint32
            lib.or_ac3.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u8p]
            lib.or_certificate.restype = ctypes.c_int64
            lib.or_certificate.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u8p]
            lib.or_peel_masked.restype = ctypes.c_uint32
            lib.or_peel_masked.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u8p, u32p, u8p]
            lib.or_scc.restype = ctypes.c_uint32
            lib.or_scc.argtypes = [ctypes.c_uint32, u32p, u32p, u32p]
            lib.or_peel_inout.restype = ctypes.c_uint32
            lib.or_peel_inout.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u32p, u32p, u8p]
            lib.or_certificate_inout.restype = ctypes.c_int64
            lib.or_certificate_inout.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u32p, u32p,
                                                 u8p]
            _lib = lib
    return _lib


def _csr(off, tgt):
    off = np.ascontiguousarray(off, np.uint32)
    tgt = np.ascontiguousarray(tgt, np.uint32)
    if tgt.size == 0:
        tgt = np.zeros(1, np.uint32)  # ctypes wants a real buffer
    return off, tgt


def transpose(off, tgt):
    """G^T as (off_in, tgt_in); predecessors listed in increasing source order."""
    off, tgt = _csr(off, tgt)
    n = off.shape[0] - 1
    off_in = np.empty(n + 1, np.uint32)
    tgt_in = np.empty(max(int(off[-1]), 1), np.uint32)
    rc = _L().or_transpose(n, off, tgt, off_in, tgt_in)
    if rc != 0:
        raise ValueError("transpose: target out of range")
    return off_in, tgt_in[:int(off[-1])]


def peel(off, tgt, csr_in=None):
    """O1 (Algorithm 5, one peeling step at a time). Returns (level, status, alpha)."""
    off, tgt = _csr(off, tgt)
    n = off.shape[0] - 1
    off_in, tgt_in = transpose(off, tgt) if csr_in is None else csr_in
    off_in, tgt_in = _csr(off_in, tgt_in)
    level = np.empty(max(n, 1), np.uint32)
    status = np.empty(max(n, 1), np.uint8)
    alpha = _L().or_peel(n, off, off_in, tgt_in, level, status)
    return level[:n], status[:n], int(alpha)


def ac6(off, tgt):
    """O2 (Algorithm 7 + levels in removal order). Returns (level, status, alpha, edges_scanned)."""
    off, tgt = _csr(off, tgt)
    n = off.shape[0] - 1
    level = np.empty(max(n, 1), np.uint32)
    status = np.empty(max(n, 1), np.uint8)
    scanned = ctypes.c_uint64(0)
    alpha = _L().or_ac6(n, off, tgt, level, status, ctypes.byref(scanned))
    return level[:n], status[:n], int(alpha), int(scanned.value)


def ac3(off, tgt):
    """O3 (Algorithm 4 with one snapshot per repetition). Returns (level, status, alpha)."""
    off, tgt = _csr(off, tgt)
    n = off.shape[0] - 1
    level = np.empty(max(n, 1), np.uint32)
    status = np.empty(max(n, 1), np.uint8)
    alpha = _L().or_ac3(n, off, tgt, level, status)
    return level[:n], status[:n], int(alpha)


def certificate(off, tgt, level, status) -> int:
    """-1 if (level, status) is the trimming result of the graph, else the first
    vertex that violates a local condition (see oracle.c)."""
    off, tgt = _csr(off, tgt)
    n = off.shape[0] - 1
    level = np.ascontiguousarray(level, np.uint32)
    status = np.ascontiguousarray(status, np.uint8)
    if n == 0:
        return -1
    return int(_L().or_certificate(n, off, tgt, level, status))


def peel_inout(off, tgt, csr_in=None):
    """In+out trimming (removal on no live successor or no live predecessor, one
    peeling step at a time; see or_peel_inout). Returns (level, status, alpha)."""
    off, tgt = _csr(off, tgt)
    n = off.shape[0] - 1
    off_in, tgt_in = transpose(off, tgt) if csr_in is None else csr_in
    off_in, tgt_in = _csr(off_in, tgt_in)
    level = np.empty(max(n, 1), np.uint32)
    status = np.empty(max(n, 1), np.uint8)
    alpha = _L().or_peel_inout(n, off, tgt, off_in, tgt_in, level, status)
    return level[:n], status[:n], int(alpha)


def certificate_inout(off, tgt, level, status, csr_in=None) -> int:
    """-1 if (level, status) is the in+out trimming result of the graph, else the
    first vertex that violates a local condition (see or_certificate_inout)."""
    off, tgt = _csr(off, tgt)
    n = off.shape[0] - 1
    if n == 0:
        return -1
    off_in, tgt_in = transpose(off, tgt) if csr_in is None else csr_in
    off_in, tgt_in = _csr(off_in, tgt_in)
    level = np.ascontiguousarray(level, np.uint32)
    status = np.ascontiguousarray(status, np.uint8)
    return int(_L().or_certificate_inout(n, off, tgt, off_in, tgt_in, level, status))


def peel_masked(off, tgt, mask, csr_in=None):
    """Trimming with the vertices where mask != 0 DEAD from the start (Section
    9's vertex sampling; see or_peel_masked). Their level is MASKED; alpha
    counts the steps that removed something. Returns (level, status, alpha)."""
    off, tgt = _csr(off, tgt)
    n = off.shape[0] - 1
    off_in, tgt_in = transpose(off, tgt) if csr_in is None else csr_in
    off_in, tgt_in = _csr(off_in, tgt_in)
    mask = np.ascontiguousarray(mask, np.uint8)
    if mask.size == 0:
        mask = np.zeros(1, np.uint8)
    level = np.empty(max(n, 1), np.uint32)
    status = np.empty(max(n, 1), np.uint8)
    alpha = _L().or_peel_masked(n, off, off_in, tgt_in, mask, level, status)
    return level[:n], status[:n], int(alpha)


def scc(off, tgt):
    """Strongly connected components (Tarjan). Returns (comp, count) with
    comp[v] = the smallest vertex id of v's component."""
    off, tgt = _csr(off, tgt)
    n = off.shape[0] - 1
    comp = np.empty(max(n, 1), np.uint32)
    k = _L().or_scc(n, off, tgt, comp)
    if k == 0xFFFFFFFF:
        raise MemoryError("or_scc: allocation failed")
    return comp[:n], int(k)
