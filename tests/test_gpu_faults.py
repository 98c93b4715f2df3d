"""Host-injected fault cases of the C ABI on the GPU: every one is a small,
well-formed launch or a host-side refusal, so none can fault the device.
Each bad input must come back as its error code, and the process (and, where
one exists, the context) must keep working afterwards."""
import numpy as np
import pytest

import graphgen as gg
import graphgen.configs as cfg
import oracle

pytestmark = pytest.mark.gpu


def _P():
    import paper_2107_12720_gb300 as P
    return P


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def create(P, off, tgt, off_in=None, tgt_in=None, flags=0):
    """trim_create on device arrays of the given contents (no host-side checks
    apply to device memory: only TRIM_FLAG_VALIDATE can see the contents)."""
    csr = P.abi.TrimCsr(len(off) - 1, len(tgt), off.data_ptr(), tgt.data_ptr(), P.TRIM_MEM_DEVICE)
    csr_in = None
    if off_in is not None:
        csr_in = P.abi.TrimCsr(len(off_in) - 1, len(tgt_in), off_in.data_ptr(), tgt_in.data_ptr(),
                               P.TRIM_MEM_DEVICE)
    return P.trim_create(csr, csr_in, None, flags)


def expect(P, code, fn, *a):
    with pytest.raises(P.TrimError) as e:
        fn(*a)
    assert e.value.code == code, (e.value.code, str(e.value))


def still_works(P):
    g = cfg.config_small(0)
    lvl, st, alpha = oracle.peel(g.off, g.tgt)
    with P.Trimmer(g.off, g.tgt) as t:
        assert t.run("ac4")["rounds"] == alpha
        assert np.array_equal(t.level(device=False), lvl)


def test_validate_rejects_non_monotone_offsets():
    P = _P()
    g = cfg.config_small(1)
    off = g.off.copy()
    off[10] = off[11] + 1  # offsets[10] > offsets[11]
    expect(P, 2, create, P, dev(off), dev(g.tgt), None, None, P.TRIM_FLAG_VALIDATE)
    still_works(P)


def test_validate_rejects_a_target_out_of_range():
    P = _P()
    g = cfg.config_small(1)
    tgt = g.tgt.copy()
    tgt[len(tgt) // 2] = g.n  # one past the last vertex
    expect(P, 2, create, P, dev(g.off), dev(tgt), None, None, P.TRIM_FLAG_VALIDATE)
    still_works(P)


def test_validate_rejects_offsets_that_do_not_end_at_m():
    P = _P()
    g = cfg.config_small(2)
    tgt = g.tgt[:-1].copy()  # m - 1 targets, offsets still end at m
    expect(P, 2, create, P, dev(g.off), dev(tgt), None, None, P.TRIM_FLAG_VALIDATE)
    still_works(P)


def test_validate_rejects_a_csr_in_that_is_not_the_transpose():
    P = _P()
    g = cfg.config_small(1)
    oi, ti = oracle.transpose(g.off, g.tgt)
    # same degrees, one edge moved to another predecessor
    ti2 = ti.copy()
    row = int(np.argmax(np.diff(oi.astype(np.int64)) >= 2))
    a = int(oi[row])
    ti2[a] = (ti2[a] + 1) % g.n
    expect(P, 2, create, P, dev(g.off), dev(g.tgt), dev(oi), dev(ti2), P.TRIM_FLAG_VALIDATE)
    # degrees that differ
    oi3 = oi.copy()
    oi3[1:-1] = oi3[2:]
    oi3[-1] = oi[-1]
    expect(P, 2, create, P, dev(g.off), dev(g.tgt), dev(oi3), dev(ti), P.TRIM_FLAG_VALIDATE)
    # the true transpose passes
    ctx = create(P, dev(g.off), dev(g.tgt), dev(oi), dev(ti), P.TRIM_FLAG_VALIDATE)
    P.trim_destroy(ctx)
    still_works(P)


def test_allocation_cap_gives_oom_and_recovers():
    P = _P()
    g = cfg.config_small(1)
    try:
        P.trim_set_alloc_limit(4096)  # far below one context's arena
        with pytest.raises(P.TrimError) as e:
            P.Trimmer(g.off, g.tgt)
        assert e.value.code == 4
    finally:
        P.trim_set_alloc_limit(0)
    still_works(P)
    # a cap that fits the arena but not the device-built G^T: the first AC-4
    # run needs more memory and fails cleanly; AC-6 needs none and still runs
    with P.Trimmer(g.off, g.tgt) as t:
        lvl, _, _ = oracle.peel(g.off, g.tgt)
        try:
            P.trim_set_alloc_limit(1)
            with pytest.raises(P.TrimError) as e:
                t.run("ac4")
            assert e.value.code == 4
        finally:
            P.trim_set_alloc_limit(0)
        t.run("ac6")
        assert np.array_equal(t.level(device=False), lvl)
        t.run("ac4")
        assert np.array_equal(t.level(device=False), lvl)


def test_calls_out_of_order_and_bad_arguments():
    P = _P()
    g = cfg.config_small(0)
    with P.Trimmer(g.off, g.tgt) as t:
        expect(P, 7, t.level, False)             # before any run: TRIM_ERR_STATE
        expect(P, 7, t.status, False)
        expect(P, 7, t.run, "scripted")          # no schedule set
        expect(P, 1, P.trim_run, t.ctx, 99)      # unknown variant
        expect(P, 1, t.batch_run, np.array([0, 5], np.uint32), "ac4")  # does not end at n
        expect(P, 1, t.batch_run, np.array([0, g.n, 3, g.n], np.uint32), "ac4")  # decreasing
        expect(P, 1, lambda: t.set_params(block_threads=100))  # not a multiple of 32
        expect(P, 1, lambda: t.set_params(spin_limit_ns=0))
        expect(P, 1, P.trim_set_model, t.ctx, np.zeros(5, np.float32))  # wrong size
        expect(P, 1, P.trim_set_schedule, t.ctx, np.array([0, 3], np.uint8))  # entry > 2
        lvl, _, alpha = oracle.peel(g.off, g.tgt)
        assert t.run("ac4")["rounds"] == alpha   # the context still works
        assert np.array_equal(t.level(device=False), lvl)
    # a closed context is refused, not dereferenced
    expect(P, 1, P.trim_run, None, 0)
    expect(P, 1, t.run, "ac4")
