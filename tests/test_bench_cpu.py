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
