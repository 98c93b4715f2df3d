"""The asynchronous AC-4 tail against the oracle.

From round 128 on, once the in-edges still to push are few (async_round_edges),
an AC-4 run finishes without rounds: each CTA pushes the rows of the vertices it
removes at its own pace, and a removed vertex takes one more than the top level
among its successors (Definition 2), carried by the pushes in a 64-bit
compare-and-swap word. Levels, status, alpha, the removal count and the pushed
in-edges must equal the oracle's (and the round-synchronous run's) bit for bit,
whatever order the pushes take. Rows longer than the shared-memory queue go to
a global list in 256-edge pieces that a rebalance spreads over all CTAs; the
graphs below force that path at every other level of a chain, and with a
100,000-in-edge hub deep in it.
"""
import numpy as np
import pytest

import graphgen as gg
import graphgen.configs as cfg
import oracle
from tests.test_gpu_parity import _confident_ac4_model, check, dev_csr, dev_csr_in, hand_cases

pytestmark = pytest.mark.gpu

ASYNC_MIN_ROUND = 128


def _P():
    import paper_2107_12720_gb300 as P
    return P


def broom(L=260, short_until=136, small=3, big=1500, mid=300, hub_at=150, hub=100_000):
    """A chain c_{L-1} -> ... -> c_0 (c_0 a sink); chain vertex c_i has k_i
    leaf predecessors (out-degree 1, into c_i): 3 for i < short_until (the
    rows pending when the tail takes over, at round 128, stay short), then
    1,500 (even i: longer than the shared-memory queue takes) or 300 (odd i),
    and 100,000 at c_hub_at. Levels: c_i = i, its leaves i + 1."""
    k = np.array([small if i < short_until else
                  (hub if i == hub_at else (big if i % 2 == 0 else mid))
                  for i in range(L)], np.int64)
    leaf_tgt = np.repeat(np.arange(L, dtype=np.uint32), k)
    n = L + leaf_tgt.size
    outdeg = np.ones(n, np.int64)
    outdeg[0] = 0
    off = np.zeros(n + 1, np.uint32)
    off[1:] = np.cumsum(outdeg)
    tgt = np.concatenate([np.arange(L - 1, dtype=np.uint32), leaf_tgt])
    return off, tgt


def _pushed(off, tgt, st):
    oi, _ = oracle.transpose(off, tgt)
    return int(np.diff(oi.astype(np.int64))[st == 0].sum())


def _check_tail(s, lvl, st, alpha, label):
    if alpha >= ASYNC_MIN_ROUND:
        assert s["async_round"] == ASYNC_MIN_ROUND, (label, s)
        assert s["async_removed"] == int(((lvl >= ASYNC_MIN_ROUND) & (st == 0)).sum()), label
    else:
        assert s["async_round"] == 0, (label, s)
    assert s["rounds_by_variant"] == [alpha, 0, 0], (label, s)


@pytest.mark.parametrize("i", [0, 1, 2, 3, 4])
def test_small_configs_async_equals_rounds(i):
    """Every small workload: the tail (default; it takes over at round 128 in
    the deep cascade and the mixed graph) and round-synchronous AC-4
    (async_round_edges = 0, with and without local rounds) give the oracle's
    levels, alpha, removal count and in-edge pushes."""
    P = _P()
    g = cfg.config_small(i)
    lvl, st, alpha = oracle.peel(g.off, g.tgt)
    want = _pushed(g.off, g.tgt, st)
    with P.Trimmer(g.off, g.tgt, flags=P.TRIM_FLAG_STATS) as t:
        s = t.run("ac4")
        check(t, lvl, st, alpha, f"async[{i}]", s)
        assert s["in_edges_pushed"] == want
        if i in (0, 2, 4):  # deep enough, short pending rows at round 8
            _check_tail(s, lvl, st, alpha, f"async[{i}]")
        for local in (1 << 18, 0):
            t.set_params(async_round_edges=0, local_round_edges=local)
            s2 = t.run("ac4")
            check(t, lvl, st, alpha, f"rounds[{i}] local={local}", s2)
            assert s2["async_round"] == 0 and s2["in_edges_pushed"] == want


@pytest.mark.parametrize("name", ["long_chain", "chain", "worked_example", "big_in_hub",
                                  "duplicates", "self_loops", "edgeless", "single"])
def test_hand_cases_async(name):
    """The hand cases (alpha below 128: rounds only) and a 300-vertex chain
    (the tail takes over at round 128, one vertex per level)."""
    P = _P()
    if name == "long_chain":
        k = 300
        g = gg.edges_from_lists(k, [[]] + [[i - 1] for i in range(1, k)])
    else:
        g = hand_cases()[name]
    lvl, st, alpha = oracle.peel(g.off, g.tgt)
    with P.Trimmer(g.off, g.tgt) as t:
        s = t.run("ac4")
        check(t, lvl, st, alpha, name, s)
        _check_tail(s, lvl, st, alpha, name)


@pytest.mark.parametrize("block", [512, 128])
def test_rows_spill_to_the_global_queue(block):
    """The broom: from c_136 on every other chain vertex has a 1,501-edge G^T
    row (beyond the shared-memory queue: 256-edge pieces in the global list,
    spread over the CTAs by a rebalance), and c_150's 100,001 in-edges become
    391 pieces. With 128
    threads per CTA the queue holds 1,024 entries, so rows spill more often."""
    P = _P()
    off, tgt = broom()
    lvl, st, alpha = oracle.peel(off, tgt)
    assert alpha == 261
    assert lvl[0] == 0 and lvl[259] == 259
    with P.Trimmer(off, tgt, flags=P.TRIM_FLAG_STATS) as t:
        t.set_params(block_threads=block)
        for rep in range(3):
            s = t.run("ac4")
            check(t, lvl, st, alpha, f"broom-{block}-{rep}", s)
            _check_tail(s, lvl, st, alpha, "broom")
            assert s["in_edges_pushed"] == off.size - 2  # every edge, once
            assert s["async_rebalances"] > 0  # the spilled rows came back through rebalances


def test_thresholds_and_repeated_runs():
    """The tail taking over later (or never) gives the same result; repeated
    runs on one context re-initialise the per-vertex words every time."""
    P = _P()
    g = cfg.config_small(2)
    lvl, st, alpha = oracle.peel(g.off, g.tgt)
    with P.Trimmer(g.off, g.tgt) as t:
        for edges in (1 << 18, 4096, 64, 1, 0):
            t.set_params(async_round_edges=edges)
            for rep in range(2):
                s = t.run("ac4")
                check(t, lvl, st, alpha, f"async{edges}-{rep}", s)
                if edges == 0:
                    assert s["async_round"] == 0
                elif s["async_round"]:
                    assert s["async_round"] >= ASYNC_MIN_ROUND
                    assert s["async_removed"] == int(((lvl >= s["async_round"]) & (st == 0)).sum())


def test_scheduled_runs_take_the_tail_inside_committed_stretches():
    """Heuristic and learned runs that commit to AC-4 take the tail inside a
    committed stretch (stretches of 64, then 128 rounds: round 128 falls in the
    second; every handover); with a round log they never do (the
    log needs rounds), and without a commit the scheduler keeps the rounds. The
    learned runs use a model that picks AC-4 with high confidence."""
    P = _P()
    for i in (2, 4):
        g = cfg.config_small(i)
        lvl, st, alpha = oracle.peel(g.off, g.tgt)
        off, tgt = dev_csr(g)
        oi, ti = dev_csr_in(g)
        for flags in (0, P.TRIM_FLAG_ROUND_LOG):
            with P.Trimmer(off, tgt, oi, ti, flags=flags) as t:
                t.set_model(_confident_ac4_model())
                for h, hv in (("device", P.TRIM_HANDOVER_DEVICE), ("host", P.TRIM_HANDOVER_HOST),
                              ("none", P.TRIM_HANDOVER_NONE)):
                    t.set_params(sched_commit_rounds=1, sched_recheck_rounds=64,
                                 sched_handover=hv)
                    for mode in ("heuristic", "learned"):
                        s = t.run(mode)
                        check(t, lvl, st, alpha, f"{mode}[{i}]-{h}-{flags}", s)
                        assert s["rounds_by_variant"] == [alpha, 0, 0]
                        if flags:
                            assert s["async_round"] == 0
                        elif h == "none":
                            assert s["async_round"] == 0  # the all-variant kernel has no tail
                        else:
                            assert s["async_round"] == ASYNC_MIN_ROUND, (mode, h, s)
                t.set_params(sched_commit_rounds=0, sched_handover=P.TRIM_HANDOVER_DEVICE)
                s = t.run("heuristic")
                check(t, lvl, st, alpha, f"uncommitted[{i}]-{flags}", s)
                assert s["async_round"] == 0


@pytest.mark.parametrize("sampled", [0.5, 0.9])
def test_dead_mask_with_the_tail(sampled):
    """Masked vertices (counter 0, never pushed) are left alone by the
    compare-and-swap pushes; levels equal the oracle's masked peeling."""
    P = _P()
    from tests.test_gpu_masked import check_masked, mask_for
    for i in (2, 4):
        g = cfg.config_small(i)
        mask = mask_for(g, sampled, 31 + i)
        with P.Trimmer(g.off, g.tgt) as t:
            t.set_dead_mask(mask)
            check_masked(t, g, mask, t.run("ac4"), f"masked-async[{i}] {sampled}")


def test_batched_run_with_the_tail():
    """Packed graphs (one launch) with the tail: the oracle's levels on the union."""
    P = _P()
    u = cfg.config_small(3)
    lvl, st, alpha = oracle.peel(u.off, u.tgt)
    with P.Trimmer(u.off, u.tgt) as t:
        t.set_params(async_round_edges=1 << 20)
        for v in ("ac4", "heuristic"):
            check(t, lvl, st, alpha, f"batch-{v}", t.batch_run(u.graph_off, v))


def test_full_deep_cascade_takes_the_tail():
    """The 2^24-vertex deep cascade (alpha 2,868) in the benchmark's launch
    shape: local rounds until round 127, the tail from round 128; the levels
    equal the oracle's."""
    P = _P()
    g = cfg.config(2)
    oi_np, ti_np = oracle.transpose(g.off, g.tgt)
    lvl, st, alpha = oracle.peel(g.off, g.tgt, (oi_np, ti_np))
    import torch
    off, tgt = dev_csr(g)
    oi = torch.from_numpy(oi_np.astype(np.int32)).cuda()
    ti = torch.from_numpy(ti_np.astype(np.int32)).cuda()
    with P.Trimmer(off, tgt, oi, ti) as t:
        s = t.run("ac4")
        check(t, lvl, st, alpha, "deep-async", s)
        _check_tail(s, lvl, st, alpha, "deep-async")
