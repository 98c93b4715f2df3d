"""G^T built on the device (trim_in_csr on a context created without csr_in)
against the oracle's transpose: the in-offsets must be equal, and every row
must hold the same predecessors (the device leaves their order within a row
unspecified, the oracle lists them in increasing order, so rows are sorted
before the comparison). The graphs cover the bucket sizes of the device build
(fewer and more than 8,192 vertices, bucket boundaries), hubs with many
in-edges (the case the build is designed for), duplicates, self-loops, empty
rows and the full-size rmat22 workload."""
import numpy as np
import pytest

import graphgen as gg
import graphgen.configs as cfg
import oracle

pytestmark = pytest.mark.gpu


def _rows_sorted(off, tgt):
    n = off.shape[0] - 1
    row = np.repeat(np.arange(n, dtype=np.int64), np.diff(off.astype(np.int64)))
    order = np.lexsort((tgt.astype(np.int64), row))
    return tgt[order]


def _check(g):
    import paper_2107_12720_gb300 as P
    want_off, want_tgt = oracle.transpose(g.off, g.tgt)
    with P.Trimmer(g.off, g.tgt) as t:
        for _ in range(2):  # a second call returns the same, kept G^T
            got_off, got_tgt = t.in_csr()
            assert np.array_equal(got_off, want_off), g.name
            assert np.array_equal(_rows_sorted(got_off, got_tgt), want_tgt), g.name
        # AC-4 runs on the G^T built here
        lvl, st, alpha = oracle.peel(g.off, g.tgt)
        s = t.run("ac4")
        assert np.array_equal(t.level(device=False), lvl) and s["rounds"] == alpha


def _random(n, m, seed, hubs=0, hub_share=0.0):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    if hubs:
        k = int(m * hub_share)
        dst[:k] = rng.integers(0, hubs, k)  # most edges into a few vertices
    order = np.argsort(src, kind="stable")
    off = np.zeros(n + 1, np.uint32)
    np.cumsum(np.bincount(src, minlength=n), out=off[1:])
    return gg.Graph(off, dst[order].astype(np.uint32), name=f"random{n}_{m}_{hubs}")


@pytest.mark.parametrize("i", [0, 1, 2, 3, 4])
def test_small_configs(i):
    _check(cfg.config_small(i))


@pytest.mark.parametrize("n", [1, 2, 31, 8191, 8192, 8193, 100_003])
def test_bucket_sizes(n):
    _check(_random(n, 5 * n, seed=n))


def test_hubs():
    # 400,000 edges, 90% of them into 3 vertices; duplicates and self-loops kept
    _check(_random(50_000, 400_000, seed=3, hubs=3, hub_share=0.9))
    rows = [[]] + [[0]] * 70_000  # one target with 70,000 predecessors
    _check(gg.edges_from_lists(70_001, rows))


def test_edgeless_and_single():
    _check(gg.edges_from_lists(9, [[]] * 9))
    _check(gg.edges_from_lists(1, [[0]]))


def test_full_rmat22():
    _check(cfg.config(1))


def test_above_2_27_vertices():
    """Graphs with more than 2^27 vertices take the direct global counting
    sort (the two-level build's per-bucket counters would not fit a CTA):
    134,217,731 vertices, 300,000 random edges, a third of them into one hub."""
    g = _random((1 << 27) + 3, 300_000, seed=27, hubs=1, hub_share=0.33)
    _check(g)


def test_widest_buckets():
    """2^26 + 1 vertices: the two-level build's widest buckets (32,768 targets,
    128 KB of counters in the placement pass), 2,000,000 edges."""
    _check(_random((1 << 26) + 1, 2_000_000, seed=26, hubs=5, hub_share=0.2))
