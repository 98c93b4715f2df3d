"""Pins of the oracle's SCC decomposition (oracle.scc, Tarjan's algorithm;
Section 1: FW-BW with trimming computes it): brute-force reachability on
every 4-vertex digraph and on random small graphs (u and v share a component
iff each reaches the other), networkx's strongly_connected_components on
larger graphs, and the trimming link: a vertex the in+out trimming removes is
a component of its own. No GPU involved."""
import numpy as np
import pytest

import graphgen as gg
import graphgen.configs as cfg
import oracle
from tests.brute import batch_to_union_csr


def brute_scc(adj):
    n = adj.shape[0]
    R = np.eye(n, dtype=bool) | adj
    for _ in range(n):  # transitive closure by repeated squaring-free propagation
        R = R | ((R.astype(np.int64) @ R.astype(np.int64)) > 0)
    same = R & R.T
    return np.array([np.nonzero(same[v])[0].min() for v in range(n)], np.uint32)


def test_all_4_vertex_digraphs():
    n = 4
    codes = np.arange(1 << (n * n), dtype=np.int64)
    adjs = ((codes[:, None] >> np.arange(n * n)) & 1).astype(bool).reshape(-1, n, n)
    want = np.concatenate([brute_scc(a) + np.uint32(i * n) for i, a in enumerate(adjs)])
    off, tgt = batch_to_union_csr(adjs)
    comp, k = oracle.scc(off, tgt)
    np.testing.assert_array_equal(comp, want)
    assert k == len(np.unique(want))


@pytest.mark.parametrize("n", [6, 10, 16])
def test_random_small_graphs(n):
    rng = np.random.default_rng(300 + n)
    for trial in range(150):
        adj = rng.random((n, n)) < rng.uniform(0.03, 0.4)
        rows = []
        for v in range(n):
            r = [int(t) for t in np.nonzero(adj[v])[0]]
            rng.shuffle(r)
            rows.append(r + r[:1])  # shuffled, one duplicate
        g = gg.edges_from_lists(n, rows)
        comp, _ = oracle.scc(g.off, g.tgt)
        np.testing.assert_array_equal(comp, brute_scc(adj))


@pytest.mark.parametrize("i", [0, 1, 2, 3])
def test_networkx_on_the_small_workloads(i):
    nx = pytest.importorskip("networkx")
    g = cfg.config_small(i)
    G = nx.DiGraph()
    G.add_nodes_from(range(g.n))
    src = np.repeat(np.arange(g.n), np.diff(g.off.astype(np.int64)))
    G.add_edges_from(zip(src.tolist(), g.tgt.tolist()))
    want = np.empty(g.n, np.uint32)
    count = 0
    for c in nx.strongly_connected_components(G):
        c = list(c)
        want[c] = min(c)
        count += 1
    comp, k = oracle.scc(g.off, g.tgt)
    np.testing.assert_array_equal(comp, want)
    assert k == count


def test_trimmed_vertices_are_singletons():
    """Section 1: the vertices in+out trimming removes are size-1 SCCs."""
    for i in [0, 1, 2, 3]:
        g = cfg.config_small(i)
        comp, _ = oracle.scc(g.off, g.tgt)
        _, st, _ = oracle.peel_inout(g.off, g.tgt)
        sizes = np.bincount(comp, minlength=g.n)
        dead = np.nonzero(st == 0)[0]
        assert (comp[dead] == dead).all() and (sizes[dead] == 1).all()


def test_figure1_components():
    """Figure 1's shape: two 3-cycles joined through v6 -> v7, a source and a
    sink attached, a lone self-loop."""
    rows = [[1], [2], [0, 3], [4], [5], [6], [7], [5, 9], [0], [], [10]]
    g = gg.edges_from_lists(11, rows)
    comp, k = oracle.scc(g.off, g.tgt)
    np.testing.assert_array_equal(comp, [0, 0, 0, 3, 4, 5, 5, 5, 8, 9, 10])
    assert k == 7
