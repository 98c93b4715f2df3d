"""The seeded input generators (graphgen) against their stated recipes: the
counter-based SplitMix64 words against the published mixing function, the
id permutations are bijections, and each workload family has the structure
its recipe states (no CPU or GPU trimming involved). A graph must not depend
on the number of generator threads."""
import os
import subprocess
import sys

import numpy as np
import pytest

import graphgen as gg
import graphgen.configs as cfg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix64(z):
    """SplitMix64's output mixing function (Steele, Lea & Flood, OOPSLA 2014)."""
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 & M64
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB & M64
    return z ^ (z >> 31)


def test_counter_generator_matches_its_definition():
    for seed, stream, i in [(0, 0, 0), (1, 2, 3), (5, 1 << 45, 12345), (M64, 7, 1 << 40)]:
        key = mix64(seed ^ mix64((stream + GAMMA) & M64))
        want = mix64((key + (i + 1) * GAMMA) & M64)
        assert gg.word(seed, stream, i) == want, (seed, stream, i)


@pytest.mark.parametrize("n", [1, 2, 7, 100, 1000, 4096])
def test_id_permutations_are_bijections(n):
    p = gg.perm(3, 11, n)
    assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint32))


def rows(g):
    for v in range(g.n):
        yield v, g.tgt[g.off[v]:g.off[v + 1]]


def test_rmat_recipe():
    g = cfg.rmat22(2, scale=12)
    n = 1 << 12
    assert g.n == n and g.m <= 16 * n and int(g.off[-1]) == g.m
    assert (g.tgt < n).all()
    deg = np.diff(g.off.astype(np.int64))
    assert (deg == 0).sum() >= n // 10          # out-edges of floor(0.1 n) vertices deleted
    for v, r in rows(g):
        assert (np.diff(r.astype(np.int64)) > 0).all(), v   # sorted, no duplicates
        assert not (r == v).any(), v                        # no self-loops
    # skewed degrees: the largest in-degree far above the mean
    indeg = np.bincount(g.tgt, minlength=n)
    assert indeg.max() > 20 * indeg.mean()
    again = cfg.rmat22(2, scale=12)
    assert np.array_equal(g.off, again.off) and np.array_equal(g.tgt, again.tgt)
    other = cfg.rmat22(3, scale=12)
    assert not np.array_equal(g.tgt[:1000], other.tgt[:1000])


def test_planted_recipe():
    nC, nR, nT, sinks = 300, 300, 400, 20
    g = cfg.planted_trim(1, nC, nR, nT, sinks)
    assert g.n == nC + nR + nT
    for v, r in rows(g):
        if v < nC:            # C: draws in C only (self-loops allowed)
            assert len(r) >= 1 and (r < nC).all(), v
        elif v < nC + nR:     # R: one edge into C, the rest in R and C
            assert (r < nC).any() and (r < nC + nR).all(), v
        else:                 # T: rank = id - (nC + nR); the lowest ranks are sinks
            rank = v - nC - nR
            if rank < sinks:
                assert len(r) == 0, v
            else:
                assert 1 <= len(r) <= 4 and (r >= nC + nR).all() and (r < v).all(), v


def test_deep_cascade_recipe():
    log2n, chains = 12, 16
    g = cfg.deep_cascade(3, log2n=log2n, n_chains=chains)
    n = 1 << log2n
    nC, nR = n // 10, n // 5
    base = nC + nR
    for v, r in rows(g):
        if v >= base:
            rank = v - base
            pos, chain = divmod(rank, chains)
            if pos == 0:
                assert len(r) == 0, v
            else:   # the predecessor link plus extras at strictly lower positions
                assert base + (pos - 1) * chains + chain in r, v
                assert len(r) <= 15 and ((r - base) // chains < pos).all() and (r >= base).all(), v


def test_batched_recipe():
    u = cfg.config_small(3)
    go = u.graph_off.astype(np.int64)
    assert go[0] == 0 and go[-1] == u.n and len(go) == 65
    sizes = np.diff(go)
    assert (sizes >= 8).all() and (sizes <= 20000).all()
    owner = np.repeat(np.arange(len(sizes)), sizes)
    src = np.repeat(np.arange(u.n), np.diff(u.off.astype(np.int64)))
    assert np.array_equal(owner[src], owner[u.tgt])      # no edge leaves its graph


def test_large_mixed_recipe():
    u = cfg.config_small(4)
    assert u.meta["rmat_n"] == 1 << 15
    nC, nR, nT, chains = u.meta["block"]
    assert nC + nR + nT == 1 << 14 and u.n == (1 << 15) + (1 << 14)
    src = np.repeat(np.arange(u.n), np.diff(u.off.astype(np.int64)))
    assert ((src < u.meta["rmat_n"]) == (u.tgt < u.meta["rmat_n"])).all()  # two disjoint parts


def test_graphs_do_not_depend_on_the_thread_count():
    code = ("import hashlib, graphgen.configs as c; g = c.rmat22(2, scale=14); "
            "h = c.deep_cascade(3, log2n=14, n_chains=32); "
            "print(hashlib.sha256(g.off.tobytes() + g.tgt.tobytes() + h.off.tobytes() "
            "+ h.tgt.tobytes()).hexdigest())")
    digests = set()
    for threads in ("1", "3", "8"):
        env = dict(os.environ, OMP_NUM_THREADS=threads, PYTHONPATH=ROOT)
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                           text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        digests.add(r.stdout.strip())
    assert len(digests) == 1


def implicit_rows(seed, salt, nC, nR, nT, c_k, r_k, t_sinks, t_k, n_chains):
    """Successor lists of the implicit planted graph as include/trim.h defines
    them (written from that definition, not from the generator's source)."""
    def word(v, i):
        key = mix64(seed ^ mix64((salt + v + GAMMA) & M64))
        return mix64((key + (i + 1) * GAMMA) & M64)

    def below(w, k):
        return (w * k) >> 64

    def draw(v, lo, hi):
        return lo + below(word(v, 0), hi - lo + 1)

    out = []
    for v in range(nC + nR + nT):
        if v < nC:
            k = draw(v, *c_k)
            succ = [below(word(v, 1 + j), nC) for j in range(k)]
        elif v < nC + nR:
            k = draw(v, *r_k)
            succ = [below(word(v, 1 + j), nC if j == 0 else nC + nR) for j in range(k)]
        else:
            rank = v - nC - nR
            if n_chains == 0:
                k = 0 if rank < t_sinks else draw(v, *t_k)
                succ = [nC + nR + below(word(v, 1 + j), rank) for j in range(k)]
            else:
                pos = rank // n_chains
                k = 0 if pos == 0 else 1 + draw(v, *t_k)
                succ = [v - n_chains if j == 0 else
                        nC + nR + below(word(v, 1 + j), pos * n_chains) for j in range(k)]
        out.append(succ)
    return out


@pytest.mark.parametrize("params", [
    dict(seed=9, salt=0, nC=50, nR=40, nT=60, c_k=(4, 4), r_k=(1, 4), t_sinks=5, t_k=(1, 4),
         n_chains=0),
    dict(seed=3, salt=123, nC=40, nR=80, nT=280, c_k=(8, 8), r_k=(1, 15), t_sinks=0,
         t_k=(0, 14), n_chains=8)])
def test_implicit_definition_equals_the_generated_graph(params):
    """The successor function that trim_create_implicit documents gives, row by
    row once sorted and deduplicated, the graph graphgen materialises for the
    oracle."""
    g = gg.planted(params["seed"], params["nC"], params["nR"], params["nT"], c_k=params["c_k"],
                   r_k=params["r_k"], t_sinks=params["t_sinks"], t_k=params["t_k"],
                   n_chains=params["n_chains"], salt=params["salt"])
    want = implicit_rows(**params)
    for v, r in rows(g):
        assert r.tolist() == sorted(set(want[v])), v
