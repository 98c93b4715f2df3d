"""Trimming an implicit graph (Section 2.1's on-the-fly property): the
library's seeded planted graph, whose successors the AC-6 and AC-3 kernels
compute instead of loading a CSR, against the oracle on the same graph
materialised by the input generators (graphgen implements the generator on
its own, from the same published definition). Duplicate successors (kept by
the implicit rows, removed by graphgen) change no level."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

CASES = {
    # planted_trim recipe at small size: C 300 / R 300 / T 400, 20 sinks
    "planted": dict(seed=1, nC=300, nR=300, nT=400, c_k=(4, 4), r_k=(1, 4), t_sinks=20,
                    t_k=(1, 4)),
    # deep cascade recipe (chains, degree-8 reading) at 2^16 vertices
    "chains": dict(seed=3, nC=6553, nR=13107, nT=45876, c_k=(8, 8), r_k=(1, 15),
                   t_k=(0, 14), n_chains=64),
    "salted": dict(seed=9, nC=1000, nR=500, nT=20000, c_k=(1, 3), r_k=(1, 2), t_sinks=300,
                   t_k=(1, 6), salt=1 << 40),
    "no_core": dict(seed=4, nC=0, nR=0, nT=5000, t_sinks=50, t_k=(1, 3)),
}


def _P():
    import paper_2107_12720_gb300 as P
    return P


def materialised(c):
    return gg.planted(c["seed"], c["nC"], c["nR"], c["nT"], c_k=c.get("c_k", (4, 4)),
                      r_k=c.get("r_k", (1, 4)), t_sinks=c.get("t_sinks", 0),
                      t_k=c.get("t_k", (1, 4)), n_chains=c.get("n_chains", 0),
                      salt=c.get("salt", 0))


@pytest.mark.parametrize("name", list(CASES))
def test_implicit_matches_the_oracle(name):
    P = _P()
    c = CASES[name]
    g = materialised(c)
    lvl, st, alpha = oracle.peel(g.off, g.tgt)
    with P.Trimmer.implicit(**c, flags=P.TRIM_FLAG_STATS) as t:
        assert t.n == g.n
        inspected = {}
        for v in ["ac6", "ac3", "ac6"]:
            s = t.run(v)
            got = t.level(device=False)
            bad = np.nonzero(got != lvl)[0]
            assert bad.size == 0, f"{name} {v}: {bad.size} levels differ"
            assert np.array_equal(t.status(device=False), st)
            assert s["rounds"] == alpha and s["n_dead"] == int((st == 0).sum())
            inspected[v] = s["edges_inspected"]
        # AC-6 inspects each computed edge at most once (Section 8); AC-3 re-inspects
        assert inspected["ac6"] <= inspected["ac3"]


def test_implicit_refuses_what_needs_edges_in_memory():
    P = _P()
    with P.Trimmer.implicit(**CASES["planted"]) as t:
        for v in ["ac4", "heuristic", "learned", "scripted"]:
            with pytest.raises(P.TrimError) as e:
                t.run(v)
            assert e.value.code == 1, v
        with pytest.raises(P.TrimError) as e:
            t.run_inout()
        assert e.value.code == 1
        with pytest.raises(P.TrimError) as e:
            t.batch_run(np.array([0, t.n], np.uint32), "ac6")
        assert e.value.code == 1
        t.set_dead_mask(np.zeros(t.n, np.uint8))
        with pytest.raises(P.TrimError) as e:
            t.run("ac6")
        assert e.value.code == 1
        t.set_dead_mask(None)
        t.run("ac6")  # still works
    bad = dict(CASES["planted"], c_k=(5, 4))
    with pytest.raises(P.TrimError) as e:
        P.Trimmer.implicit(**bad)
    assert e.value.code == 1


def test_implicit_deep_cascade_full_size():
    """The deep cascade recipe at full size (2^24 vertices, ~1.4e8 computed
    edges) with AC-6: every vertex against the oracle on the materialised graph."""
    P = _P()
    n = 1 << 24
    nC, nR = n // 10, n // 5
    c = dict(seed=3, nC=nC, nR=nR, nT=n - nC - nR, c_k=(8, 8), r_k=(1, 15), t_k=(0, 14),
             n_chains=4096)
    g = materialised(c)
    lvl, st, alpha = oracle.peel(g.off, g.tgt)
    with P.Trimmer.implicit(**c) as t:
        s = t.run("ac6")
        assert np.array_equal(t.level(device=False), lvl)
        assert s["rounds"] == alpha
