"""SCC decomposition on the GPU (trim_run_scc: in+out trimming, size-2
trimming, colour-partitioned FW-BW) against the oracle's Tarjan labels,
element by element: hand cases, random multigraphs, every small workload,
the full-size workloads, and the work counters."""
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


def check_scc(t, g, label, device=False):
    want, k = oracle.scc(g.off, g.tgt)
    comp, st = t.run_scc(device=device)
    if device:
        comp = comp.cpu().numpy().view(np.uint32)
    bad = np.nonzero(comp != want)[0]
    assert bad.size == 0, f"{label}: {bad.size} labels differ, first {bad[:5]} got " \
                          f"{comp[bad[:5]]} want {want[bad[:5]]}"
    assert st["components"] == k, (label, st["components"], k)
    _, io_st, _ = oracle.peel_inout(g.off, g.tgt)
    assert st["trimmed_size1"] == int((io_st == 0).sum()), label
    return st


def figure1():
    rows = [[1], [2], [0, 3], [4], [5], [6], [7], [5, 9], [0], [], [10]]
    return gg.edges_from_lists(11, rows)


@pytest.mark.parametrize("name", list(hand_cases().keys()) + ["figure1"])
def test_hand_cases(name):
    P = _P()
    g = figure1() if name == "figure1" else hand_cases()[name]
    with P.Trimmer(g.off, g.tgt) as t:
        check_scc(t, g, name)


def test_size2_components_and_partitions():
    """Mutual pairs closed on one side are size-2 components found by step 2;
    pairs with a way out are found by FW-BW; vertices between two large
    components (Figure 1's v6, v7) come out as singletons after FW-BW removes
    the large ones."""
    P = _P()
    rows = []
    # 100 closed 2-cycles (0<->1, 2<->3, ...), the second half with an extra in-edge from a source
    for i in range(100):
        rows += [[2 * i + 1], [2 * i]]
    src = len(rows)
    rows.append([2 * i for i in range(50, 100)])  # a source into the second half
    # 2-cycles entered from a 3-cycle X and leaving to a 3-cycle Y: closed on
    # neither side, so only FW-BW separates them
    x0 = len(rows) + 40
    y0 = x0 + 3
    for i in range(20):
        a = len(rows)
        rows += [[a + 1, y0], [a]]
    rows += [[x0 + 1] + [x0 - 40 + 2 * i for i in range(20)], [x0 + 2], [x0]]  # X -> every pair
    rows += [[y0 + 1], [y0 + 2], [y0]]                                          # Y
    g = gg.edges_from_lists(len(rows), rows)
    with P.Trimmer(g.off, g.tgt) as t:
        st = check_scc(t, g, "pairs")
        assert st["trimmed_size2"] >= 100
        assert st["fwbw_steps"] >= 1


def test_random_multigraphs():
    P = _P()
    rng = np.random.default_rng(17)
    for trial in range(10):
        n = int(rng.integers(20, 4000))
        m = int(rng.integers(0, 3 * n))
        src = np.sort(rng.integers(0, n, m))
        dst = rng.integers(0, n, m)
        off = np.zeros(n + 1, np.uint32)
        np.add.at(off, src + 1, 1)
        g = gg.Graph(np.cumsum(off).astype(np.uint32), dst.astype(np.uint32))
        with P.Trimmer(g.off, g.tgt) as t:
            check_scc(t, g, f"random {trial}", device=bool(trial % 2))


@pytest.mark.parametrize("i", [0, 1, 2, 3, 4])
def test_small_configs(i):
    P = _P()
    g = cfg.config_small(i)
    with P.Trimmer(g.off, g.tgt) as t:
        check_scc(t, g, f"config_small({i})")
        # the context still trims afterwards
        lvl, _, alpha = oracle.peel(g.off, g.tgt)
        assert t.run("ac4")["rounds"] == alpha
        assert np.array_equal(t.level(device=False), lvl)
        check_scc(t, g, "again")


@pytest.mark.parametrize("i", [0, 1, 2, 3])
def test_full_configs(i):
    P = _P()
    g = cfg.config(i)
    off, tgt = dev_csr(g)
    with P.Trimmer(off, tgt) as t:
        check_scc(t, g, f"config({i})", device=True)
