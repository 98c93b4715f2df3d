"""CPU-side checks of the boundary: the library loads without a GPU, exports
every function include/trim.h declares, and rejects bad arguments on the host
before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "trim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(trim_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_12720_gb300 import build
    build.build()
    import paper_2107_12720_gb300 as P
    return P.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_binding_declares_every_header_symbol(lib):
    from paper_2107_12720_gb300.abi import SIGNATURES
    bound = {s[0] for s in SIGNATURES}
    assert set(declared_functions()) == bound


def test_struct_layouts_match_header(lib, tmp_path):
    """Size and every field offset of the binding's structs equal what a C
    compiler makes of include/trim.h."""
    import subprocess
    from paper_2107_12720_gb300.abi import (TrimCsr, TrimImplicitGraph, TrimParams, TrimRoundRec,
                                            TrimRunStats, TrimSccStats)
    structs = {"trim_csr_t": TrimCsr, "trim_params_t": TrimParams,
               "trim_run_stats_t": TrimRunStats, "trim_round_rec_t": TrimRoundRec,
               "trim_implicit_graph_t": TrimImplicitGraph, "trim_scc_stats_t": TrimSccStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "trim.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(root, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln.strip())}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_host_argument_checks_without_device(lib):
    import paper_2107_12720_gb300 as P
    from paper_2107_12720_gb300.abi import TrimCsr
    ctx = ctypes.c_void_p()
    # null csr
    assert lib.trim_create(None, None, None, 0, ctypes.byref(ctx)) == 1
    off = np.array([0, 1, 2], np.uint32)
    tgt = np.array([1, 0], np.uint32)
    csr = TrimCsr(2, 2, off.ctypes.data, tgt.ctypes.data, 0)
    # unknown flag bits
    assert lib.trim_create(ctypes.byref(csr), None, None, 0x80, ctypes.byref(ctx)) == 1
    # m too large for uint32 offsets
    big = TrimCsr(2, 1 << 33, off.ctypes.data, tgt.ctypes.data, 0)
    assert lib.trim_create(ctypes.byref(big), None, None, 0, ctypes.byref(ctx)) == 3
    # limits that keep every index computation from wrapping: n <= 2^31, m <= 2^32 - 64
    big = TrimCsr((1 << 31) + 1, 2, off.ctypes.data, tgt.ctypes.data, 0)
    assert lib.trim_create(ctypes.byref(big), None, None, 0, ctypes.byref(ctx)) == 3
    big = TrimCsr(2, (1 << 32) - 63, off.ctypes.data, tgt.ctypes.data, 0)
    assert lib.trim_create(ctypes.byref(big), None, None, 0, ctypes.byref(ctx)) == 3
    # offsets inconsistent with m (host check)
    bad = TrimCsr(2, 3, off.ctypes.data, tgt.ctypes.data, 0)
    assert lib.trim_create(ctypes.byref(bad), None, None, 0, ctypes.byref(ctx)) == 2
    assert "offsets" in lib.trim_last_error(None).decode()
    # unknown memory kind
    odd = TrimCsr(2, 2, off.ctypes.data, tgt.ctypes.data, 7)
    assert lib.trim_create(ctypes.byref(odd), None, None, 0, ctypes.byref(ctx)) == 1
    # csr_in of a different size
    cin = TrimCsr(3, 2, off.ctypes.data, tgt.ctypes.data, 0)
    assert lib.trim_create(ctypes.byref(csr), ctypes.byref(cin), None, 0, ctypes.byref(ctx)) == 1
    # null context calls
    assert lib.trim_run(None, 0, None) == 1
    assert lib.trim_status(None, None, 0) == 1
    assert lib.trim_level(None, None, 0) == 1
    p = P.abi.TrimParams()
    assert lib.trim_default_params(ctypes.byref(p)) == 0
    assert p.block_threads == 512 and p.spin_limit_ns > 0


def test_no_device_is_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2107_12720_gb300.abi import TrimCsr
    off = np.array([0, 1, 1], np.uint32)
    tgt = np.array([1], np.uint32)
    csr = TrimCsr(2, 1, off.ctypes.data, tgt.ctypes.data, 0)
    ctx = ctypes.c_void_p()
    rc = lib.trim_create(ctypes.byref(csr), None, None, 0, ctypes.byref(ctx))
    assert rc == 8, rc  # TRIM_ERR_NO_DEVICE


def test_atomic_probe_rejects_bad_args(lib):
    ms = ctypes.c_float()
    assert lib.trim_probe_atomic_rate(None, 1, None, 1, 1, None, ctypes.byref(ms)) == 1
    buf = (ctypes.c_uint32 * 4)()
    assert lib.trim_probe_atomic_rate(buf, 0, buf, 4, 1, None, ctypes.byref(ms)) == 1
    assert lib.trim_probe_atomic_rate(buf, 4, buf, 4, 0, None, ctypes.byref(ms)) == 1


def test_mlp_entry_points_reject_bad_args(lib):
    assert lib.trim_mlp_forward(None, None, 0, None, None) == 1
    assert lib.trim_mlp_loss_grad(None, None, None, 0, None, None, None, None) == 1
    assert lib.trim_mlp_adam_step(None, None, None, None, 0, 0.0, 0.0, 0.0, 0.0, None) == 1
    assert lib.trim_mlp_scratch_bytes(1000) > 0


def test_header_constants_match_binding():
    """#define values of include/trim.h that the binding mirrors."""
    import re
    from paper_2107_12720_gb300 import abi
    hdr = open(os.path.join(ROOT, "include", "trim.h")).read()
    defs = dict(re.findall(r"#define (TRIM_[A-Z0-9_]+) \(?([0-9xA-Fa-f]+)u?", hdr))
    for name in ["TRIM_MEM_HOST", "TRIM_MEM_DEVICE", "TRIM_MEM_HOST_MAPPED", "TRIM_FLAG_VALIDATE",
                 "TRIM_FLAG_STATS", "TRIM_FLAG_ROUND_LOG", "TRIM_LIVE", "TRIM_MASKED"]:
        assert int(defs[name], 0) == getattr(abi, name), name
