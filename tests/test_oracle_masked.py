"""Pins of the oracle's vertex-sampled trimming (oracle.peel_masked): the
unsampled vertices (mask != 0) are DEAD from the start, as in the scalability
experiment of Section 9 (Figs. 7-9 sample 10%..100% of the vertices).

Pins, none of them a restatement of its algorithm:
  * deleting the unsampled vertices (with all their edges) and trimming what
    is left with walk-length brute force gives the sampled vertices' levels;
  * the same, on larger graphs, with the pinned O1 oracle on the induced
    subgraph (relabelled to 0..|S|-1);
  * an empty mask reproduces O1, a full mask leaves nothing to trim;
  * the trimmed share grows as fewer vertices are sampled (Section 9: "the
    smaller ratio of sampling ... leads to the higher ratio of trimmable
    vertices").
No GPU involved."""
import numpy as np
import pytest

import graphgen as gg
import graphgen.configs as cfg
import oracle
from tests.brute import LIVE, brute_levels

MASKED = 0xFFFFFFFE


def induced(g, mask):
    """The subgraph induced by the sampled vertices, relabelled in id order,
    and the old ids of its vertices."""
    keep = np.nonzero(mask == 0)[0]
    new = np.full(g.n, -1, np.int64)
    new[keep] = np.arange(keep.size)
    rows = []
    for v in keep:
        t = g.tgt[g.off[v]:g.off[v + 1]]
        rows.append([int(new[x]) for x in t if mask[x] == 0])
    return gg.edges_from_lists(keep.size, rows), keep


def test_brute_force_on_small_random_graphs():
    rng = np.random.default_rng(61)
    for trial in range(300):
        n = int(rng.integers(1, 11))
        adj = rng.random((n, n)) < rng.uniform(0.05, 0.5)
        mask = (rng.random(n) < rng.uniform(0.0, 0.9)).astype(np.uint8)
        rows = [[int(t) for t in np.nonzero(adj[v])[0]] for v in range(n)]
        g = gg.edges_from_lists(n, rows)
        lvl, st, alpha = oracle.peel_masked(g.off, g.tgt, mask)
        sub = adj[np.ix_(mask == 0, mask == 0)]
        want_sub = brute_levels(sub) if sub.size else np.zeros(0, np.uint32)
        want = np.full(n, MASKED, np.uint32)
        want[mask == 0] = want_sub
        np.testing.assert_array_equal(lvl, want)
        np.testing.assert_array_equal(st, (want == LIVE).astype(np.uint8))
        dead = want_sub[want_sub != LIVE]
        assert alpha == (int(dead.max()) + 1 if dead.size else 0)


@pytest.mark.parametrize("i", [0, 1, 2, 3])
@pytest.mark.parametrize("ratio", [0.1, 0.5, 0.9])
def test_induced_subgraph_on_workloads(i, ratio):
    g = cfg.config_small(i)
    rng = np.random.default_rng(int(ratio * 100) + i)
    mask = (rng.random(g.n) >= ratio).astype(np.uint8)  # ratio = share of sampled vertices
    lvl, st, alpha = oracle.peel_masked(g.off, g.tgt, mask)
    h, keep = induced(g, mask)
    wl, ws, wa = oracle.peel(h.off, h.tgt)
    np.testing.assert_array_equal(lvl[keep], wl)
    assert (lvl[mask != 0] == MASKED).all() and (st[mask != 0] == 0).all()
    assert alpha == wa


def test_empty_and_full_masks():
    g = cfg.config_small(1)
    a = oracle.peel_masked(g.off, g.tgt, np.zeros(g.n, np.uint8))
    b = oracle.peel(g.off, g.tgt)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[2] == b[2]
    lvl, st, alpha = oracle.peel_masked(g.off, g.tgt, np.ones(g.n, np.uint8))
    assert (lvl == MASKED).all() and alpha == 0 and (st == 0).all()


def test_trimmed_share_grows_as_fewer_vertices_are_sampled():
    g = cfg.config_small(1)
    rng = np.random.default_rng(3)
    u = rng.random(g.n)
    shares = []
    for ratio in (1.0, 0.7, 0.4, 0.1):
        mask = (u >= ratio).astype(np.uint8)
        lvl, st, _ = oracle.peel_masked(g.off, g.tgt, mask)
        sampled = mask == 0
        shares.append(float((st[sampled] == 0).mean()))
    assert all(a <= b for a, b in zip(shares, shares[1:])), shares
