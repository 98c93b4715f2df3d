"""Brute-force trimming for tiny graphs, independent of any peeling algorithm.

It uses walk lengths only: with A the 0/1 adjacency matrix of an n-vertex
graph, a vertex has a walk of length n iff it reaches a directed cycle (a walk
of n edges repeats a vertex; a reachable cycle gives walks of every length).
Such vertices are exactly the ones kept by Definition 1. For every other vertex
all walks are finite, and its peeling step of Definition 2 (counted from 0) is
the length of its longest walk, i.e. the largest k with row v of A^k nonzero.
"""
import numpy as np

LIVE = 0xFFFFFFFF


def brute_levels(adj):
    """adj: bool array (..., n, n). Returns uint32 levels (..., n)."""
    adj = np.asarray(adj, dtype=bool)
    n = adj.shape[-1]
    A = adj.astype(np.int64)
    P = np.broadcast_to(np.eye(n, dtype=np.int64), adj.shape).copy()  # A^0
    longest = np.zeros(adj.shape[:-1], np.int64)
    for k in range(1, n + 1):
        P = np.minimum(P @ A, 1)
        has = P.any(axis=-1)
        longest = np.where(has, k, longest)
    level = np.where(longest >= n, LIVE, longest).astype(np.uint32)
    return level


def adj_to_csr(adj):
    """bool (n,n) -> (off, tgt) with successors in increasing order."""
    adj = np.asarray(adj, dtype=bool)
    n = adj.shape[0]
    off = np.zeros(n + 1, np.uint32)
    off[1:] = np.cumsum(adj.sum(axis=1))
    tgt = np.nonzero(adj)[1].astype(np.uint32)
    return off, tgt


def batch_to_union_csr(adjs):
    """bool (G,n,n) -> union CSR of G disjoint n-vertex graphs (ids g*n+v)."""
    adjs = np.asarray(adjs, dtype=bool)
    G, n, _ = adjs.shape
    flat = adjs.reshape(G * n, n)
    deg = flat.sum(axis=1)
    off = np.zeros(G * n + 1, np.uint64)
    off[1:] = np.cumsum(deg)
    rows, cols = np.nonzero(flat)
    tgt = (rows // n) * n + cols
    return off.astype(np.uint32), tgt.astype(np.uint32)
