"""In+out trimming on the GPU (trim_run_inout) against the oracle's
peel_inout, element by element: hand cases, the small workloads (with G^T
given and built on the device), the full-size workloads, every launch shape,
work counters, and alternation with one-sided runs on the same context."""
import numpy as np
import pytest

import graphgen as gg
import graphgen.configs as cfg
import oracle
from tests.test_gpu_parity import dev_csr, hand_cases

pytestmark = pytest.mark.gpu


def _P():
    import paper_2107_12720_gb300 as P
    return P


def check_io(t, g, stats=None, csr_in=None, label=""):
    want_l, want_s, alpha = oracle.peel_inout(g.off, g.tgt, csr_in)
    lvl = t.level(device=False)
    st = t.status(device=False)
    bad = np.nonzero(lvl != want_l)[0]
    assert bad.size == 0, f"{label}: {bad.size} levels differ, first {bad[:5]} " \
                          f"got {lvl[bad[:5]]} want {want_l[bad[:5]]}"
    assert np.array_equal(st, want_s), label
    if stats is not None:
        assert stats["rounds"] == alpha, (label, stats["rounds"], alpha)
        assert stats["n_dead"] == int((want_s == 0).sum()), label


def figure1_graph():
    rows = [[1], [2], [0, 3], [4], [5], [6], [7], [5, 9], [0], [], [10]]
    return gg.edges_from_lists(11, rows)


@pytest.mark.parametrize("name", list(hand_cases().keys()) + ["figure1"])
def test_hand_cases(name):
    P = _P()
    g = figure1_graph() if name == "figure1" else hand_cases()[name]
    with P.Trimmer(g.off, g.tgt) as t:
        check_io(t, g, t.run_inout(), label=name)


@pytest.mark.parametrize("i", [0, 1, 2, 3, 4])
def test_small_configs(i):
    P = _P()
    g = cfg.config_small(i)
    oi, ti = oracle.transpose(g.off, g.tgt)
    with P.Trimmer(g.off, g.tgt, oi, ti, flags=P.TRIM_FLAG_STATS) as t:
        s = t.run_inout()
        check_io(t, g, s, (oi, ti), f"config_small({i})")
        # work: every removed vertex pushes its whole G^T row and its whole G row
        _, st, _ = oracle.peel_inout(g.off, g.tgt, (oi, ti))
        dead = st == 0
        assert s["in_edges_pushed"] == int(np.diff(oi.astype(np.int64))[dead].sum())
        assert s["edges_inspected"] == int(np.diff(g.off.astype(np.int64))[dead].sum())
        check_io(t, g, t.run_inout(), (oi, ti), "repeat")
    with P.Trimmer(g.off, g.tgt) as t:  # G^T built on the device
        check_io(t, g, t.run_inout(), None, f"config_small({i}) device G^T")


def test_alternating_with_one_sided_runs():
    """The same context runs one-sided trimming and in+out trimming in turn;
    every run resets its state and gives its own oracle's answer. G^T is built
    on the device by the first run, so it sits next to the context's other
    arrays: a run that wrote past one of them would corrupt it."""
    P = _P()
    g = cfg.config_small(2)
    lv1, st1, a1 = oracle.peel(g.off, g.tgt)
    with P.Trimmer(g.off, g.tgt) as t:
        for v in ["inout", "ac4", "inout", "ac6", "inout", "learned", "inout", "ac4"]:
            if v == "inout":
                check_io(t, g, t.run_inout(), label="alternating")
            else:
                s = t.run(v)
                assert np.array_equal(t.level(device=False), lv1), v
                assert s["rounds"] == a1


@pytest.mark.parametrize("block,cps", [(256, 0), (384, 0), (512, 1), (128, 1)])
def test_launch_shapes(block, cps):
    P = _P()
    g = cfg.config_small(1)
    with P.Trimmer(g.off, g.tgt) as t:
        t.set_params(block_threads=block, ctas_per_sm=cps)
        check_io(t, g, t.run_inout(), label=f"{block}x{cps}")


def test_random_multigraphs():
    P = _P()
    rng = np.random.default_rng(13)
    for trial in range(8):
        n = int(rng.integers(50, 3000))
        m = int(rng.integers(0, 4 * n))
        src = np.sort(rng.integers(0, n, m))
        dst = rng.integers(0, n, m)
        off = np.zeros(n + 1, np.uint32)
        np.add.at(off, src + 1, 1)
        g = gg.Graph(np.cumsum(off).astype(np.uint32), dst.astype(np.uint32))
        with P.Trimmer(g.off, g.tgt) as t:
            check_io(t, g, t.run_inout(), label=f"random {trial}")


@pytest.mark.parametrize("i", [0, 1, 2, 3])
def test_full_configs(i):
    """Full-size workloads (planted 1e5, R-MAT scale 22, deep cascade 2^24, the
    batched union of 4,096 graphs) with G^T given, every vertex compared."""
    P = _P()
    g = cfg.config(i)
    oi, ti = gg.transpose(g.off, g.tgt)
    off, tgt = dev_csr(g)
    import torch
    d_oi = torch.from_numpy(oi.view(np.int32)).cuda()
    d_ti = torch.from_numpy(ti.view(np.int32)).cuda()
    with P.Trimmer(off, tgt, d_oi, d_ti) as t:
        check_io(t, g, t.run_inout(), (oi, ti), f"config({i})")
