"""trim_run_ac4_noalloc: the entry point for callers that cannot allocate device
memory when they need a result (it takes its scratch from a fixed array inside
the library). Its levels must equal those of the allocating entry point
(trim_run with TRIM_AC4_PUSH) bit for bit, on consecutive calls that reuse the
same scratch, and sizes beyond its fixed capacity must be refused up front.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import graphgen.configs as cfg

pytestmark = pytest.mark.gpu


def transpose_np(off, tgt):
    n = off.shape[0] - 1
    src = np.repeat(np.arange(n, dtype=np.uint32), np.diff(off.astype(np.int64)))
    order = np.argsort(tgt, kind="stable")
    off_in = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(tgt, minlength=n), out=off_in[1:])
    return off_in.astype(np.uint32), src[order].astype(np.uint32)


def on_device(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()
            for a in arrays]


def levels_with_allocating_entry_point(g):
    import paper_2107_12720_gb300 as P
    with P.Trimmer(g.off, g.tgt) as t:
        stats = t.run("ac4")
        return t.level(device=False), stats["rounds"]


def levels_without_allocation(g, d_off, d_tgt, d_ioff, d_itgt, tail=0):
    """Levels from the entry point that allocates nothing. The output buffer is
    poisoned (every level must be written) and, with tail > 0, has `tail` extra
    poisoned entries after the n levels that must stay untouched."""
    import torch
    import paper_2107_12720_gb300 as P
    out = torch.full((g.n + tail,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rounds = P.abi.trim_run_ac4_noalloc(d_off, d_tgt, d_ioff, d_itgt, g.n, g.m, out, stream)
    got = out.cpu().numpy().view(np.uint32)
    if tail:
        assert (got[g.n:] == np.uint32(0xFFFFFFF9)).all(), "wrote past level_out[n)"
    return got[:g.n], rounds


def test_no_alloc_entry_point_matches_trim_run_on_consecutive_calls():
    graphs = [cfg.config_small(1), cfg.config_small(2), cfg.config_small(0),
              gg.edges_from_lists(6, [[1], [2], [0], [4], [0], [2]])]
    for g in graphs:
        assert g.n <= (1 << 18) and g.m <= (1 << 22)
        want, want_rounds = levels_with_allocating_entry_point(g)
        ioff, itgt = transpose_np(g.off, g.tgt)
        dev = on_device(g.off, g.tgt, ioff, itgt)
        for call in range(2):  # the second call reuses the scratch the first left behind
            got, rounds = levels_without_allocation(g, *dev)
            bad = np.nonzero(got != want)[0]
            assert bad.size == 0, f"{g}: call {call}: {bad.size} levels differ"
            assert rounds == want_rounds


def test_no_alloc_entry_point_at_its_size_limit():
    """A graph with exactly the largest vertex count the scratch holds (2^18)
    and close to the largest edge count (an R-MAT of scale 18 with edge factor
    16: 2^22 draws before self-loops, duplicates and sinks are dropped), so that
    every scratch region is used up to its end; level_out has a poisoned tail."""
    g = gg.rmat(11, 18, 16, 0.57, 0.19, 0.19, 0.1, name="rmat18")
    assert g.n == (1 << 18) and 0.8 * (1 << 22) < g.m <= (1 << 22)
    want, want_rounds = levels_with_allocating_entry_point(g)
    ioff, itgt = transpose_np(g.off, g.tgt)
    dev = on_device(g.off, g.tgt, ioff, itgt)
    for call in range(2):
        got, rounds = levels_without_allocation(g, *dev, tail=64)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, f"call {call}: {bad.size} levels differ"
        assert rounds == want_rounds


def test_no_alloc_entry_point_refuses_sizes_beyond_its_scratch():
    import paper_2107_12720_gb300 as P
    lib = P.lib()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    r = ctypes.c_uint32(0)
    too_many_vertices = lib.trim_run_ac4_noalloc(dummy, dummy, dummy, dummy, (1 << 18) + 1, 10,
                                                 dummy, ctypes.byref(r), None)
    too_many_edges = lib.trim_run_ac4_noalloc(dummy, dummy, dummy, dummy, 10, (1 << 22) + 1,
                                              dummy, ctypes.byref(r), None)
    assert too_many_vertices == 3 and too_many_edges == 3  # TRIM_ERR_TOO_LARGE
