"""Host-side pieces of bench.py that decide what its JSON line reports: the
algorithmic-byte model, the kernel-source key of the committed ncu summary
(comments must not orphan it; code must), and which run the traffic figure
may be attached to. No device needed."""
import os
import shutil

import bench


def test_algorithmic_bytes_model():
    st = {"n_dead": 10, "in_edges_pushed": 100, "live_swept": 7, "candidates": 3,
          "edges_inspected": 50}
    # init 12n, 20 per removed vertex, 12 per pushed in-edge, 16 per swept entry,
    # 24 per AC-6 candidate, 8 per inspected out-edge
    assert bench.algorithmic_bytes(1000, st, {}) == 12 * 1000 + 20 * 10 + 12 * 100 + 16 * 7 + 24 * 3 + 8 * 50


def test_kernel_key_ignores_comments_but_not_code(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    shutil.copy(bench.KERNEL_SRC, src)
    monkeypatch.setattr(bench, "KERNEL_SRC", str(src))
    base = bench.kernel_source_sha()
    text = src.read_text()
    src.write_text(text + "\n// a new comment line\n\n")
    assert bench.kernel_source_sha() == base
    src.write_text(text + "\nint an_extra_symbol;\n")
    assert bench.kernel_source_sha() != base


def test_traffic_only_for_the_profiled_run():
    # the committed summary covers the rmat22 workload with fixed AC-4
    assert bench.profiled_traffic(2, False, "ac4") is None
    assert bench.profiled_traffic(1, True, "ac4") is None
    assert bench.profiled_traffic(1, False, "learned") is None
    t = bench.profiled_traffic(1, False, "ac4")
    assert t is None or t > 0


def test_reference_arm_keeps_the_graph_and_caps_the_steps():
    # requested steps that fit the budget are all timed
    assert bench.reference_steps(1.0, 20, 5, 150.0) == (4, 20)
    # a slow graph: fewer timed steps, never zero, and no extra warm-up
    assert bench.reference_steps(4.0, 20, 5, 150.0) == (4, 20)
    assert bench.reference_steps(10.0, 20, 5, 150.0) == (0, 15)
    assert bench.reference_steps(500.0, 20, 5, 150.0) == (0, 1)


def test_touched_bytes_of_in_place_inputs():
    st = {"in_edges_pushed": 100, "edges_inspected": 7}
    assert bench.touched_input_bytes(10, st) == 8 * 11 + 4 * 100 + 4 * 7


def test_input_transpose_equals_the_oracles():
    """The G^T the workloads supply (graphgen, parallel) is the same array pair
    as the oracle's own transpose, duplicates and empty rows included."""
    import numpy as np
    import graphgen as gg
    import graphgen.configs as cfg
    import oracle
    graphs = [cfg.config_small(i) for i in range(4)]
    graphs.append(gg.edges_from_lists(5, [[1, 1, 1], [2, 2], [], [3, 0, 0], [4]]))
    for g in graphs:
        a, b = gg.transpose(g.off, g.tgt), oracle.transpose(g.off, g.tgt)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), g


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle timed on the host cores, no GPU
    needed) prints exactly one JSON line with the keys the benchmark contract
    asks of that arm, on the workload it was given."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "0",
                        "--steps", "3", "--warmup", "1"], cwd=root, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 1
    assert d["unit"] == "edges/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["n"] == 100000 and d["config"]["workload"].startswith("planted_trim")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "edges/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_measured_peak_or_fallback(tmp_path):
    good = tmp_path / "good.json"
    good.write_text('{"hbm_gbs": 6777.6, "bf16_tflops": 1900}')
    assert bench.measured_peaks(str(good)) == (6777.6, "measured")
    for text in ['{"bf16_tflops": 1900}', '{"hbm_gbs": null}', '{"hbm_gbs": 0}', "not json"]:
        bad = tmp_path / "bad.json"
        bad.write_text(text)
        assert bench.measured_peaks(str(bad)) == (6800.0, "fallback"), text
    assert bench.measured_peaks(str(tmp_path / "absent.json")) == (6800.0, "fallback")
