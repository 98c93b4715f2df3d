"""The autotuner's search and bookkeeping (paper_2107_12720_gb300.autotune) on a
fake context whose run time is a known function of the parameters: it must
return the minimum of the search space, keep the defaults when nothing is
faster, and round-trip its result file. No device needed."""
import os

import pytest

from paper_2107_12720_gb300 import autotune as A


class FakeTrimmer:
    def __init__(self, cost):
        self.cost = cost
        self.p = A.default_params()

    def set_params(self, **kw):
        self.p.update(kw)

    def run(self, variant):
        return {"device_ms": self.cost(variant, self.p)}


@pytest.fixture
def lib_available():
    from paper_2107_12720_gb300 import abi
    try:
        abi.lib()
    except Exception as e:  # the library is built by build(); tests that need it skip
        pytest.skip(f"libtrim.so not loadable: {e}")


def test_tune_finds_the_minimum(lib_available):
    def cost(v, p):
        c = 1.0 + abs(p["block_threads"] - 384) / 1000 + 0.1 * p["ctas_per_sm"]
        c += 0.05 * (p["local_round_edges"] != (1 << 14))
        if v == "heuristic":
            c += abs(p["heur_push_ratio"] - 2.0) + abs(p["sched_commit_rounds"] - 32) / 100
        return c
    t = FakeTrimmer(cost)
    res = A.tune(t, variants=("ac4", "heuristic"), reps=1)
    assert res["ac4"]["params"] == {"block_threads": 384, "ctas_per_sm": 0,
                                    "local_round_edges": 1 << 14}
    hp = res["heuristic"]["params"]
    assert hp["heur_push_ratio"] == 2.0 and hp["sched_commit_rounds"] == 32
    assert hp["block_threads"] == 384 and hp["local_round_edges"] == 1 << 14
    assert res["heuristic"]["ms"] < res["heuristic"]["default_ms"]


def test_defaults_kept_when_nothing_is_faster(lib_available):
    t = FakeTrimmer(lambda v, p: 1.0)
    res = A.tune(t, variants=("ac6",), reps=1)
    assert res["ac6"]["params"] == {} and res["ac6"]["ms"] == 1.0


def test_result_file_round_trip(tmp_path, lib_available):
    path = os.path.join(tmp_path, "tuned.json")
    A.save({"config1/ac4": {"params": {"block_threads": 256}, "ms": 1.0, "default_ms": 2.0}}, path)
    A.save({"config2/ac4": {"params": {}, "ms": 3.0, "default_ms": 3.0}}, path)
    t = FakeTrimmer(lambda v, p: 1.0)
    assert A.apply(t, "config1", "ac4", path) == {"block_threads": 256}
    assert t.p["block_threads"] == 256
    assert A.apply(t, "config2", "ac4", path) == {}
    assert A.apply(t, "config9", "ac4", path) == {}
