"""Named synthetic workloads.

They stand in for the paper's graphs (Section 9, Table 10: BEEM, SNAP, KONECT,
NetworkRepository and SNAP ER/BA/R-MAT at 1M vertices / 8M edges), none of which
ships here. Each keeps the shape parameters that matter for trimming: skewed
R-MAT degrees, a large trimmable share, and deep peeling (alpha in the
thousands, cf. Definition 2 and alpha up to 11.7K in Table 10).

  planted_trim      n=100,000: C 30,000 / R 30,000 / T 40,000 (2,000 sinks)
  rmat22            R-MAT scale 22, edge factor 16, (a,b,c)=(.57,.19,.19), 10% sinks
  deep_cascade      n=2^24: C 10% / R 20% / T 70% as 4,096 chains (~2,867 deep)
  batched           4,096 planted graphs, log-normal sizes, packed with graph offsets
  large_mixed       R-MAT scale 26 union a 2^25-vertex planted block with ~10,000-deep chains

Small variants (``*_small``) keep the recipe at sizes the oracle finishes in
well under a second; they are the parity-test cases.
"""
from __future__ import annotations

import numpy as np

from . import Graph, normal12, planted, rmat, union, unit, word, det_exp


def planted_trim(seed: int = 1, nC=30000, nR=30000, nT=40000, t_sinks=2000) -> Graph:
    g = planted(seed, nC, nR, nT, c_k=(4, 4), r_k=(1, 4), t_sinks=t_sinks, t_k=(1, 4),
                name=f"planted_trim(n={nC + nR + nT},seed={seed})")
    return g


def rmat22(seed: int = 2, scale: int = 22) -> Graph:
    return rmat(seed, scale, 16, 0.57, 0.19, 0.19, 0.1, name=f"rmat{scale}(seed={seed})")


def deep_cascade(seed: int = 3, log2n: int = 24, n_chains: int = 4096, literal=False) -> Graph:
    """Core 10%, reaching 20%, trimmable 70% as chains (rank = pos*n_chains+chain).

    Degree reading (mean out-degree 8): C draws 8 targets in C; R draws 1+U{0..14}
    (first in C); each chain link has its predecessor edge plus U{0..14} extra
    targets at strictly lower positions. ``literal=True`` keeps the smaller degrees
    of the planted_trim recipe instead (C 4; R 1..4; 0..3 extras), m ~ 2.6 n.
    """
    n = 1 << log2n
    nC, nR = n // 10, n // 5
    nT = n - nC - nR
    if literal:
        ck, rk, tk = (4, 4), (1, 4), (0, 3)
    else:
        ck, rk, tk = (8, 8), (1, 15), (0, 14)
    return planted(seed, nC, nR, nT, c_k=ck, r_k=rk, t_k=tk, n_chains=n_chains,
                   name=f"deep_cascade(2^{log2n},chains={n_chains}{',literal' if literal else ''})")


def batched_graph_params(seed: int, G: int, median=2000.0, sigma=1.5, nmin=64, nmax=2_000_000):
    """Per-graph (n_g, d, t) of the batched workload: n_g log-normal (median,
    sigma) clipped to [nmin,nmax], d ~ U{2..12}, t ~ U[0,0.9)."""
    out = []
    for g in range(G):
        z = normal12(seed, (1 << 50) + g)
        ng = int(round(median * det_exp(sigma * z)))
        ng = max(nmin, min(nmax, ng))
        d = 2 + (word(seed, (1 << 51) + g, 0) * 11 >> 64)
        t = 0.9 * unit(seed, (1 << 51) + g, 1)
        out.append((ng, int(d), t))
    return out


def batched(seed: int = 4, G: int = 4096, median=2000.0, sigma=1.5, nmin=64,
            nmax=2_000_000) -> Graph:
    """Disjoint union of G planted graphs (the planted_trim recipe per graph):
    |T| = floor(t n_g), |C| = max(1, floor((n_g-|T|)/2)), R the rest, the lowest
    ceil(5%) of T ranks are sinks, every other vertex draws k ~ U{1..2d-1}."""
    parts = []
    live = []
    for gi, (ng, d, t) in enumerate(batched_graph_params(seed, G, median, sigma, nmin, nmax)):
        nT = int(t * ng)
        nC = max(1, (ng - nT) // 2)
        nR = ng - nT - nC
        sinks = -(-nT * 5 // 100) if nT else 0
        k = (1, 2 * d - 1)
        g = planted(seed, nC, nR, nT, c_k=k, r_k=k, t_sinks=sinks, t_k=k, salt=gi << 40,
                    name=f"batch[{gi}]")
        parts.append(g)
        live.append(nC + nR)
    u = union(parts, name=f"batched(G={G},seed={seed})")
    u.meta = dict(seed=seed, G=G, live_per_graph=np.asarray(live, np.int64),
                  sizes=[(p.meta["nC"], p.meta["nR"], p.meta["nT"], p.meta["t_sinks"])
                         for p in parts])
    return u


def large_mixed(seed: int = 5, scale: int = 26, block_log2: int = 25, chain_len=10_000):
    """R-MAT (rmat22 recipe at ``scale``) union a planted block of 2^block_log2
    vertices: C 10%, R 20%, T 70% as chains of length ~chain_len, degree-8 reading."""
    r = rmat(seed, scale, 16, 0.57, 0.19, 0.19, 0.1, name=f"rmat{scale}")
    nb = 1 << block_log2
    nC, nR = nb // 10, nb // 5
    nT = nb - nC - nR
    chains = max(1, nT // chain_len)
    p = planted(seed, nC, nR, nT, c_k=(8, 8), r_k=(1, 15), t_k=(0, 14), n_chains=chains,
                salt=1 << 45, name="planted-block")
    u = union([r, p], name=f"large_mixed(rmat{scale}+2^{block_log2})")
    u.meta = dict(seed=seed, rmat_n=r.n, block=(nC, nR, nT, chains))
    return u


# The five named workloads, by index (0 small planted, 1 R-MAT, 2 deep, 3 batched, 4 large)
def config(i: int) -> Graph:
    return [planted_trim, rmat22, deep_cascade, batched, large_mixed][i]()


# Scaled-down variants with the same recipes: parity-test cases.
def config_small(i: int) -> Graph:
    if i == 0:
        return planted_trim(1, 300, 300, 400, 20)
    if i == 1:
        return rmat22(2, scale=14)
    if i == 2:
        return deep_cascade(3, log2n=16, n_chains=64)
    if i == 3:
        return batched(4, G=64, median=200.0, nmin=8, nmax=20000)
    if i == 4:
        return large_mixed(5, scale=15, block_log2=14, chain_len=300)
    raise ValueError(i)
