"""Seeded synthetic graphs (CSR, uint32) for the trimming library and its oracle.

This package draws graphs only; it contains none of the trimming arithmetic.
The C core (``graphgen.c``) is compiled on first use with gcc into
``libgraphgen.so`` next to it. See ``configs.py`` for the named workloads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile libgraphgen.so (gcc, OpenMP, no FP contraction) if stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-std=gnu11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class PlantedParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint32) for k in
                ("nC", "nR", "nT", "c_kmin", "c_kmax", "r_kmin", "r_kmax", "t_sinks",
                 "t_kmin", "t_kmax", "n_chains")]


class RmatParams(ctypes.Structure):
    _fields_ = [("scale", ctypes.c_int), ("ndraws", ctypes.c_uint64), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("c", ctypes.c_double), ("sink_frac", ctypes.c_double)]


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
            lib.gg_planted_maxm.restype = ctypes.c_uint64
            lib.gg_planted_maxm.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.POINTER(PlantedParams)]
            lib.gg_planted.restype = ctypes.c_uint64
            lib.gg_planted.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.POINTER(PlantedParams), u32p, u32p]
            lib.gg_rmat.restype = ctypes.c_uint64
            lib.gg_rmat.argtypes = [ctypes.c_uint64, ctypes.POINTER(RmatParams), u32p, u32p]
            lib.gg_er.restype = ctypes.c_uint64
            lib.gg_er.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, u32p, u32p]
            lib.gg_relabel.restype = None
            lib.gg_relabel.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u32p, u32p]
            lib.gg_transpose.restype = ctypes.c_int
            lib.gg_transpose.argtypes = [ctypes.c_uint32, u32p, u32p, u32p, u32p]
            lib.gg_word.restype = ctypes.c_uint64
            lib.gg_word.argtypes = [ctypes.c_uint64] * 3
            lib.gg_perm.restype = ctypes.c_uint32
            lib.gg_perm.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                    ctypes.c_uint32]
            lib.gg_exp.restype = ctypes.c_double
            lib.gg_exp.argtypes = [ctypes.c_double]
            lib.gg_unit.restype = ctypes.c_double
            lib.gg_unit.argtypes = [ctypes.c_uint64] * 3
            lib.gg_normal12.restype = ctypes.c_double
            lib.gg_normal12.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            _lib = lib
    return _lib


class Graph:
    """A directed graph in CSR: ``off`` (n+1) and ``tgt`` (m), both uint32.

    ``parts`` optionally records named vertex ranges (e.g. the C/R/T sets of a
    planted graph) and ``graph_off`` the per-graph vertex offsets of a batch.
    """

    def __init__(self, off, tgt, name="", parts=None, graph_off=None, meta=None):
        self.off = np.ascontiguousarray(off, dtype=np.uint32)
        self.tgt = np.ascontiguousarray(tgt, dtype=np.uint32)
        self.name = name
        self.parts = parts or {}
        self.graph_off = None if graph_off is None else np.ascontiguousarray(graph_off, np.uint32)
        self.meta = meta or {}

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.tgt.shape[0])

    def __repr__(self):
        return f"Graph({self.name!r}, n={self.n}, m={self.m})"


def planted(seed: int, nC: int, nR: int, nT: int, c_k=(4, 4), r_k=(1, 4), t_sinks=0,
            t_k=(1, 4), n_chains=0, salt: int = 0, name="planted") -> Graph:
    """Planted-trim graph: core C, reaching set R, trimmable set T (see graphgen.c)."""
    p = PlantedParams(nC, nR, nT, c_k[0], c_k[1], r_k[0], r_k[1], t_sinks, t_k[0], t_k[1],
                      n_chains)
    if nC == 0 and (nR > 0):
        raise ValueError("R needs a non-empty C")
    lib = _L()
    n = nC + nR + nT
    maxm = lib.gg_planted_maxm(seed, salt, ctypes.byref(p))
    off = np.empty(n + 1, np.uint32)
    tgt = np.empty(max(int(maxm), 1), np.uint32)
    m = lib.gg_planted(seed, salt, ctypes.byref(p), off, tgt)
    if m == 2**64 - 1:
        raise MemoryError("gg_planted: allocation failed")
    tgt = tgt[:m].copy() if m < tgt.shape[0] // 2 else tgt[:m]
    parts = {"C": (0, nC), "R": (nC, nC + nR), "T": (nC + nR, n)}
    return Graph(off, tgt, name, parts,
                 meta=dict(seed=seed, nC=nC, nR=nR, nT=nT, t_sinks=t_sinks, n_chains=n_chains))


def rmat(seed: int, scale: int, edge_factor: int = 16, a=0.57, b=0.19, c=0.19,
         sink_frac=0.1, name="rmat") -> Graph:
    """R-MAT graph with permuted ids, no self-loops, no duplicates, and
    floor(sink_frac*n) vertices whose out-edges are deleted."""
    n = 1 << scale
    ndraws = edge_factor * n
    p = RmatParams(scale, ndraws, a, b, c, sink_frac)
    off = np.empty(n + 1, np.uint32)
    tgt = np.empty(ndraws, np.uint32)
    m = _L().gg_rmat(seed, ctypes.byref(p), off, tgt)
    if m == 2**64 - 1:
        raise MemoryError("gg_rmat: allocation failed")
    tgt = tgt[:m].copy() if m < ndraws // 2 else tgt[:m]
    return Graph(off, tgt, name, meta=dict(seed=seed, scale=scale, edge_factor=edge_factor))


def er(seed: int, n: int, m_draws: int, name="er") -> Graph:
    """Erdos-Renyi digraph: m_draws uniform pairs without self-loops, deduplicated."""
    off = np.empty(n + 1, np.uint32)
    tgt = np.empty(max(m_draws, 1), np.uint32)
    m = _L().gg_er(seed, n, m_draws, off, tgt)
    if m == 2**64 - 1:
        raise MemoryError("gg_er failed")
    return Graph(off, tgt[:m], name, meta=dict(seed=seed))


def perm(seed: int, salt: int, n: int) -> np.ndarray:
    """A pseudo-random bijection of [0,n) as an array (perm[old] = new)."""
    lib = _L()
    return np.fromiter((lib.gg_perm(seed, salt, n, i) for i in range(n)), np.uint32, n)


def relabel(g: Graph, p: np.ndarray, name=None) -> Graph:
    """Relabel vertex v as p[v]; rows stay sorted."""
    p = np.ascontiguousarray(p, np.uint32)
    off2 = np.empty_like(g.off)
    tgt2 = np.empty_like(g.tgt) if g.m else np.empty(1, np.uint32)
    _L().gg_relabel(g.n, g.off, g.tgt if g.m else np.empty(1, np.uint32), p, off2, tgt2)
    return Graph(off2, tgt2[:g.m], name or g.name + "-relabelled", meta=dict(g.meta))


def union(graphs, name="union") -> Graph:
    """Disjoint union: graph i's ids are shifted by the vertex count before it.
    Returns a Graph whose ``graph_off`` holds the per-graph vertex offsets."""
    ns = [g.n for g in graphs]
    vo = np.zeros(len(graphs) + 1, np.int64)
    vo[1:] = np.cumsum(ns)
    eo = np.zeros(len(graphs) + 1, np.int64)
    eo[1:] = np.cumsum([g.m for g in graphs])
    if vo[-1] >= 2**32 - 1 or eo[-1] >= 2**32:
        raise ValueError("union too large for uint32 CSR")
    off = np.empty(vo[-1] + 1, np.uint32)
    tgt = np.empty(eo[-1], np.uint32)
    for i, g in enumerate(graphs):
        off[vo[i]:vo[i + 1]] = g.off[:-1] + np.uint32(eo[i])
        tgt[eo[i]:eo[i + 1]] = g.tgt + np.uint32(vo[i])
    off[-1] = np.uint32(eo[-1])
    return Graph(off, tgt, name, graph_off=vo.astype(np.uint32))


def transpose(off, tgt):
    """G^T of a CSR graph as (off_in, tgt_in), rows in ascending source order:
    the in-CSR the workloads supply next to the out-CSR (input preparation,
    parallel; the oracle keeps its own transpose)."""
    off = np.ascontiguousarray(off, np.uint32)
    tgt = np.ascontiguousarray(tgt, np.uint32)
    n = off.shape[0] - 1
    m = int(off[-1]) if n >= 0 else 0
    off_in = np.empty(n + 1, np.uint32)
    tgt_in = np.empty(max(m, 1), np.uint32)
    rc = _L().gg_transpose(n, off, tgt if tgt.size else np.zeros(1, np.uint32), off_in, tgt_in)
    if rc == -1:
        raise ValueError("transpose: target out of range")
    if rc != 0:
        raise MemoryError("transpose: allocation failed")
    return off_in, tgt_in[:m]


def word(seed: int, stream: int, i: int) -> int:
    return int(_L().gg_word(seed, stream, i))


def unit(seed: int, stream: int, i: int) -> float:
    return float(_L().gg_unit(seed, stream, i))


def normal12(seed: int, stream: int) -> float:
    return float(_L().gg_normal12(seed, stream))


def det_exp(x: float) -> float:
    return float(_L().gg_exp(x))


def edges_from_lists(n: int, adj) -> Graph:
    """Small hand-built graph from a list of successor lists (kept in the given
    order; duplicates and self-loops are kept as given)."""
    off = np.zeros(n + 1, np.uint32)
    flat = []
    for v in range(n):
        succ = list(adj[v]) if v < len(adj) else []
        flat.extend(succ)
        off[v + 1] = off[v] + len(succ)
    return Graph(off, np.asarray(flat, np.uint32), "hand")
