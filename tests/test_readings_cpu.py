"""CPU checks of two readings the kernels rely on, each against facts that do
not come from the kernels: brute force over walk lengths on small graphs and
the oracle's peel on the small workloads. No GPU involved.

Levels without rounds (Definition 2 read as a recurrence): once every push
carries the level of the vertex it comes from, and each predecessor keeps the
largest level pushed so far beside its counter of live successors, the push
that takes the counter to zero fixes the level as that maximum + 1, whatever
order the pushes arrive in. The model below applies the pushes one at a time
in random orders (each one indivisible, as a compare-and-swap on a 64-bit word
makes it), optionally after some synchronous rounds (the hand-over from
rounds to the asynchronous tail) and with vertex-sampling masks.

AC-3 "change" semantics (Section 4, Algorithm 4): a sweep that reads the
statuses it is updating (Gauss-Seidel) removes the same vertices as sweeps
over snapshots (Jacobi, the oracle's O3), in at most as many sweeps."""
import numpy as np
import pytest

import graphgen as gg
import graphgen.configs as cfg
import oracle
from tests.brute import LIVE, adj_to_csr, brute_levels

MASKED = oracle.MASKED


def predecessors(off, tgt):
    """One entry per edge copy: u appears in preds[w] once per edge u -> w."""
    n = len(off) - 1
    preds = [[] for _ in range(n)]
    for u in range(n):
        for e in range(int(off[u]), int(off[u + 1])):
            preds[int(tgt[e])].append(u)
    return preds


def levels_by_unordered_pushes(off, tgt, rng, sync_rounds=0, mask=None):
    """Levels from pushes applied in a random order. The first `sync_rounds`
    peeling steps run as synchronous rounds; the pushes of the last frontier
    and of everything removed after it are then applied one at a time, each
    picked at random from all pending pushes."""
    n = len(off) - 1
    preds = predecessors(off, tgt)
    masked = np.zeros(n, bool) if mask is None else np.asarray(mask, bool)
    # live-successor counters over unmasked successors; a masked vertex keeps 0
    cnt = [0 if masked[u] else sum(1 for e in range(int(off[u]), int(off[u + 1]))
                                   if not masked[int(tgt[e])]) for u in range(n)]
    level = [MASKED if masked[u] else LIVE for u in range(n)]
    frontier = [u for u in range(n) if not masked[u] and cnt[u] == 0]
    for u in frontier:
        level[u] = 0
    r = 1
    while r <= sync_rounds and frontier:
        nxt = []
        for w in frontier:
            for u in preds[w]:
                if cnt[u] == 0:
                    continue  # masked: pushes leave it alone
                cnt[u] -= 1
                if cnt[u] == 0:
                    level[u] = r
                    nxt.append(u)
        frontier, r = nxt, r + 1
    top = [0] * n  # largest level pushed so far, beside the counter
    pending = [(u, level[w]) for w in frontier for u in preds[w]]
    while pending:
        i = int(rng.integers(len(pending)))
        pending[i], pending[-1] = pending[-1], pending[i]
        u, lw = pending.pop()
        if cnt[u] == 0:
            assert masked[u], "a push reached a vertex that was already removed"
            continue
        top[u] = max(top[u], lw)
        cnt[u] -= 1
        if cnt[u] == 0:
            level[u] = top[u] + 1
            pending.extend((p, level[u]) for p in preds[u])
    return np.array(level, np.uint32)


def random_adjacency(rng, n):
    p = rng.uniform(0.05, 0.5)
    return rng.random((n, n)) < p


@pytest.mark.parametrize("n", [5, 8, 12])
def test_unordered_pushes_give_the_walk_length_levels(n):
    rng = np.random.default_rng(1000 + n)
    for _ in range(120):
        adj = random_adjacency(rng, n)
        off, tgt = adj_to_csr(adj)
        want = brute_levels(adj)
        for sync_rounds in (0, 1, 3):
            got = levels_by_unordered_pushes(off, tgt, rng, sync_rounds)
            assert np.array_equal(got, want), (adj.astype(int), sync_rounds)


def test_unordered_pushes_on_multigraphs_and_the_small_workloads():
    rng = np.random.default_rng(7)
    graphs = [gg.edges_from_lists(5, [[1, 1, 1], [2, 2], [], [3, 0, 0], [4]]),
              gg.edges_from_lists(6, [[1], [2], [0], [4], [0], [2]])]
    graphs += [cfg.config_small(i) for i in (0, 2)]
    for g in graphs:
        want, _, _ = oracle.peel(g.off, g.tgt)
        for sync_rounds in (0, 2, 5):
            got = levels_by_unordered_pushes(g.off, g.tgt, rng, sync_rounds)
            bad = np.nonzero(got != want)[0]
            assert bad.size == 0, (g, sync_rounds, bad[:5])


def test_unordered_pushes_with_sampled_vertices():
    """Masked vertices keep counter 0 and are skipped by pushes; the levels
    equal the oracle's vertex-sampled trimming."""
    rng = np.random.default_rng(11)
    g = cfg.config_small(2)
    for ratio in (0.3, 0.7):
        mask = (rng.random(g.n) < ratio).astype(np.uint8)
        want, _, _ = oracle.peel_masked(g.off, g.tgt, mask)
        got = levels_by_unordered_pushes(g.off, g.tgt, rng, 2, mask)
        assert np.array_equal(got, want), ratio


def test_a_dropped_maximum_is_caught():
    """The model is sensitive to the recurrence: keeping the first pushed level
    instead of the largest gives wrong levels on some graph here."""
    rng = np.random.default_rng(3)

    def first_level_only(off, tgt):
        n = len(off) - 1
        preds = predecessors(off, tgt)
        cnt = [int(off[u + 1] - off[u]) for u in range(n)]
        level = [LIVE] * n
        first = [None] * n
        pending = []
        for u in range(n):
            if cnt[u] == 0:
                level[u] = 0
                pending.extend((p, 0) for p in preds[u])
        while pending:
            i = int(rng.integers(len(pending)))
            pending[i], pending[-1] = pending[-1], pending[i]
            u, lw = pending.pop()
            first[u] = lw if first[u] is None else first[u]
            cnt[u] -= 1
            if cnt[u] == 0:
                level[u] = first[u] + 1
                pending.extend((p, level[u]) for p in preds[u])
        return np.array(level, np.uint32)

    caught = False
    for _ in range(200):
        adj = random_adjacency(rng, 8)
        off, tgt = adj_to_csr(adj)
        if not np.array_equal(first_level_only(off, tgt), brute_levels(adj)):
            caught = True
            break
    assert caught


def gauss_seidel_ac3(off, tgt):
    """Algorithm 4 with in-place statuses: a vertex removed earlier in the same
    sweep already counts as removed. Returns (status, sweeps that removed)."""
    n = len(off) - 1
    live = [True] * n
    sweeps = 0
    while True:
        change = False
        for v in range(n):
            if live[v] and not any(live[int(tgt[e])] for e in range(int(off[v]), int(off[v + 1]))):
                live[v] = False
                change = True
        if not change:
            return np.array(live, np.uint8), sweeps
        sweeps += 1


@pytest.mark.parametrize("n", [6, 10])
def test_in_place_ac3_sweeps_keep_the_status_in_at_most_alpha_sweeps(n):
    rng = np.random.default_rng(500 + n)
    fewer = 0
    for _ in range(150):
        adj = random_adjacency(rng, n)
        off, tgt = adj_to_csr(adj)
        want = brute_levels(adj)
        alpha = int(want[want != LIVE].max()) + 1 if (want != LIVE).any() else 0
        status, sweeps = gauss_seidel_ac3(off, tgt)
        assert np.array_equal(status, (want == LIVE).astype(np.uint8))
        assert sweeps <= alpha
        fewer += sweeps < alpha
    assert fewer > 0  # in-place sweeps do take fewer sweeps on some graphs
