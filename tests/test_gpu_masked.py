"""Vertex-sampled trimming on the GPU (trim_set_dead_mask): every variant and
schedule, batched runs, host and device masks, against the oracle's
peel_masked element by element, for sampled shares of 10%..90% (Section 9's
scalability experiment samples vertices by setting the unsampled ones DEAD)."""
import numpy as np
import pytest

import graphgen.configs as cfg
import oracle
from tests.test_gpu_parity import dev_csr, dev_csr_in

pytestmark = pytest.mark.gpu

VARIANTS = ["ac4", "ac6", "ac3", "heuristic", "learned"]


def _P():
    import paper_2107_12720_gb300 as P
    return P


def mask_for(g, sampled, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(g.n) >= sampled).astype(np.uint8)


def check_masked(t, g, mask, stats, label):
    want_l, want_s, alpha = oracle.peel_masked(g.off, g.tgt, mask)
    lvl = t.level(device=False)
    st = t.status(device=False)
    bad = np.nonzero(lvl != want_l)[0]
    assert bad.size == 0, f"{label}: {bad.size} levels differ, first {bad[:5]} got " \
                          f"{lvl[bad[:5]]} want {want_l[bad[:5]]}"
    assert np.array_equal(st, want_s), label
    assert stats["rounds"] == alpha, (label, stats["rounds"], alpha)
    trimmed = int(((want_s == 0) & (mask == 0)).sum())
    assert stats["n_dead"] == trimmed, (label, stats["n_dead"], trimmed)


@pytest.mark.parametrize("i", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("sampled", [0.1, 0.5, 0.9])
def test_small_configs_every_variant(i, sampled):
    P = _P()
    from paper_2107_12720_gb300 import scheduler
    g = cfg.config_small(i)
    mask = mask_for(g, sampled, 7 * i + int(sampled * 10))
    off, tgt = dev_csr(g)
    oi, ti = dev_csr_in(g)
    with P.Trimmer(off, tgt, oi, ti) as t:
        t.set_model(scheduler.load_blob())
        t.set_dead_mask(mask)
        for v in VARIANTS:
            check_masked(t, g, mask, t.run(v), f"config_small({i}) {sampled} {v}")


def test_device_mask_batches_and_clearing():
    """A mask given in device memory, a batched run under a mask, and clearing
    the mask (the next run is the unmasked trimming again)."""
    import torch
    P = _P()
    u = cfg.config_small(3)
    mask = mask_for(u, 0.6, 3)
    with P.Trimmer(u.off, u.tgt) as t:
        t.set_dead_mask(torch.from_numpy(mask).cuda())
        for v in ["ac4", "ac4", "ac6"]:  # the second call replays a captured graph
            check_masked(t, u, mask, t.batch_run(u.graph_off, v), f"batch {v}")
        t.set_dead_mask(None)
        lvl, st, alpha = oracle.peel(u.off, u.tgt)
        s = t.run("ac4")
        assert np.array_equal(t.level(device=False), lvl) and s["rounds"] == alpha


def test_all_masked_and_none_masked():
    P = _P()
    g = cfg.config_small(1)
    with P.Trimmer(g.off, g.tgt) as t:
        for mask in (np.ones(g.n, np.uint8), np.zeros(g.n, np.uint8)):
            t.set_dead_mask(mask)
            for v in ["ac4", "ac6", "ac3"]:
                check_masked(t, g, mask, t.run(v), f"{int(mask[0])} {v}")


def test_inout_refuses_a_mask():
    P = _P()
    g = cfg.config_small(0)
    with P.Trimmer(g.off, g.tgt) as t:
        t.set_dead_mask(mask_for(g, 0.5, 1))
        with pytest.raises(P.TrimError) as e:
            t.run_inout()
        assert e.value.code == 1
        t.set_dead_mask(None)
        t.run_inout()  # the context still works


@pytest.mark.parametrize("sampled", [0.1, 0.3, 0.5, 0.7, 0.9])
def test_full_rmat22_sampled(sampled):
    """The R-MAT scale-22 workload with vertex samples of 10%..90% (the
    paper's scalability experiment on a synthetic stand-in), every fixed
    variant and the learned schedule, every vertex compared."""
    P = _P()
    from paper_2107_12720_gb300 import scheduler
    g = cfg.config(1)
    mask = mask_for(g, sampled, 100 + int(sampled * 10))
    off, tgt = dev_csr(g)
    oi, ti = dev_csr_in(g)
    with P.Trimmer(off, tgt, oi, ti) as t:
        t.set_model(scheduler.load_blob())
        t.set_dead_mask(mask)
        for v in ["ac4", "ac6", "ac3", "learned"]:
            check_masked(t, g, mask, t.run(v), f"rmat22 {sampled} {v}")
