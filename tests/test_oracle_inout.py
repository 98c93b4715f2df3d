"""Pins of the oracle's in+out trimming (oracle.peel_inout): removal when a
vertex has no live successor OR no live predecessor (Section 4's remark on
checking the in-degree when G^T is loaded; the size-1 SCC trimming of FW-BW and
ISPAN, Section 1), one peeling step at a time.

What pins it, none of it a restatement of its algorithm:
  * status: a vertex survives iff it reaches a directed cycle AND is reached
    from one (walks of length n forward and backward, tests/brute.py);
  * levels: the in+out level of every vertex is min(a, b), where a is its
    Definition-2 level in G and b its Definition-2 level in G^T (both from
    walk-length brute force). min(a, b) satisfies the local certificate
    (level = min(t_out, t_in), see or_certificate_inout), and the certificate
    holds for exactly one assignment;
  * the certificate itself rejects mutated answers;
  * the process is symmetric: G and G^T give the same result;
  * the paper's Figure 1 situation: vertices between two large SCCs are
    size-1 SCCs that in+out trimming cannot remove.
No GPU involved."""
import numpy as np
import pytest

import graphgen as gg
import graphgen.configs as cfg
import oracle
from tests.brute import LIVE, adj_to_csr, batch_to_union_csr, brute_levels


def brute_inout(adjs):
    """min(level in G, level in G^T) by walk lengths (LIVE = 0xFFFFFFFF is the max)."""
    adjs = np.asarray(adjs, dtype=bool)
    return np.minimum(brute_levels(adjs), brute_levels(np.swapaxes(adjs, -1, -2)))


def cycle_status(adj):
    """1 iff the vertex reaches a cycle and a cycle reaches it (walks of length n)."""
    n = adj.shape[-1]
    A = adj.astype(np.int64)
    F = np.eye(n, dtype=np.int64)
    B = np.eye(n, dtype=np.int64)
    for _ in range(n):
        F = np.minimum(F @ A, 1)
        B = np.minimum(B @ A.T, 1)
    return (F.any(axis=1) & B.any(axis=1)).astype(np.uint8)


def test_all_4_vertex_digraphs():
    """Every digraph on 4 vertices (self-loops included), as one disjoint union."""
    n = 4
    codes = np.arange(1 << (n * n), dtype=np.int64)
    adjs = ((codes[:, None] >> np.arange(n * n)) & 1).astype(bool).reshape(-1, n, n)
    want = brute_inout(adjs).reshape(-1)
    off, tgt = batch_to_union_csr(adjs)
    lvl, st, alpha = oracle.peel_inout(off, tgt)
    np.testing.assert_array_equal(lvl, want)
    np.testing.assert_array_equal(st, (want == LIVE).astype(np.uint8))
    assert alpha == int(want[want != LIVE].max()) + 1
    assert oracle.certificate_inout(off, tgt, lvl, st) == -1


@pytest.mark.parametrize("n", [5, 8, 12])
def test_random_small_graphs_and_cycle_status(n):
    rng = np.random.default_rng(200 + n)
    for trial in range(120):
        adj = rng.random((n, n)) < rng.uniform(0.02, 0.45)
        want = brute_inout(adj)
        rows = []
        for v in range(n):
            r = [int(t) for t in np.nonzero(adj[v])[0]]
            rng.shuffle(r)
            if r and rng.random() < 0.4:
                r = r + r[:1]  # a duplicate edge
            rows.append(r)
        g = gg.edges_from_lists(n, rows)
        lvl, st, _ = oracle.peel_inout(g.off, g.tgt)
        np.testing.assert_array_equal(lvl, want)
        np.testing.assert_array_equal(st, cycle_status(adj))


def test_symmetric_under_reversal():
    for i in [0, 1, 2, 3]:
        g = cfg.config_small(i)
        oi, ti = oracle.transpose(g.off, g.tgt)
        a = oracle.peel_inout(g.off, g.tgt, (oi, ti))
        b = oracle.peel_inout(oi, ti, (g.off, g.tgt))
        np.testing.assert_array_equal(a[0], b[0])
        assert a[2] == b[2]


def test_min_of_the_two_one_sided_trimmings_on_the_workloads():
    """On the small workloads (too large for walk-length brute force) the in+out
    levels equal min(Definition-2 levels of G, of G^T), with the one-sided
    levels from the pinned O1 oracle."""
    for i in [0, 1, 2, 3, 4]:
        g = cfg.config_small(i)
        oi, ti = oracle.transpose(g.off, g.tgt)
        lv, st, _ = oracle.peel_inout(g.off, g.tgt, (oi, ti))
        a = oracle.peel(g.off, g.tgt, (oi, ti))[0]
        b = oracle.peel(oi, ti, (g.off, g.tgt))[0]
        np.testing.assert_array_equal(lv, np.minimum(a, b))
        assert oracle.certificate_inout(g.off, g.tgt, lv, st, (oi, ti)) == -1


def test_figure1_vertices_between_two_sccs_stay():
    """Section 1, Figure 1: v6 and v7 between two large SCCs are size-1 SCCs
    that trimming cannot remove directly; the tails hanging off the SCCs go.
    Here SCC1 = {0,1,2} (a 3-cycle) -> 3 (v6) -> 4 (v7) -> SCC2 = {5,6,7};
    8 -> 0 has no predecessor, 7 -> 9 has no successor, 10 -> 10 is a lone
    self-loop (a size-1 SCC that is not trimmable)."""
    rows = [[1], [2], [0, 3], [4], [5], [6], [7], [5, 9], [0], [], [10]]
    g = gg.edges_from_lists(11, rows)
    lvl, st, alpha = oracle.peel_inout(g.off, g.tgt)
    want_status = np.array([1, 1, 1, 1, 1, 1, 1, 1, 0, 0, 1], np.uint8)
    np.testing.assert_array_equal(st, want_status)
    assert lvl[8] == 0 and lvl[9] == 0 and alpha == 1
    # out-only trimming keeps the source 8 (it reaches a cycle)
    assert oracle.peel(g.off, g.tgt)[1][8] == 1


def test_certificate_rejects_mutations():
    g = cfg.config_small(2)
    oi, ti = oracle.transpose(g.off, g.tgt)
    lvl, st, _ = oracle.peel_inout(g.off, g.tgt, (oi, ti))
    assert oracle.certificate_inout(g.off, g.tgt, lvl, st, (oi, ti)) == -1
    rng = np.random.default_rng(9)
    dead = np.nonzero(st == 0)[0]
    live = np.nonzero(st == 1)[0]
    for trial in range(24):
        l2, s2 = lvl.copy(), st.copy()
        kind = trial % 4
        if kind == 0:
            v = rng.choice(dead)
            l2[v] += 1
        elif kind == 1:
            v = rng.choice(dead[lvl[dead] > 0])
            l2[v] -= 1
        elif kind == 2:
            v = rng.choice(dead)
            l2[v], s2[v] = LIVE, 1
        else:
            v = rng.choice(live)
            l2[v], s2[v] = 0, 0
        assert oracle.certificate_inout(g.off, g.tgt, l2, s2, (oi, ti)) != -1
    # the out-only answer is not an in+out answer on this graph (sources exist)
    lo, so, _ = oracle.peel(g.off, g.tgt, (oi, ti))
    assert oracle.certificate_inout(g.off, g.tgt, lo, so, (oi, ti)) != -1
