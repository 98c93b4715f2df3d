"""The C ABI from plain C99: tests/c/trim_c_client.c is compiled with gcc
against include/trim.h and linked to libtrim.so. On a machine without a GPU it
must get TRIM_ERR_NO_DEVICE (no CPU fallback); on a GB300 it trims a chain and a
2-cycle with every variant."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "trim_c_client.c")
LIBDIR = os.path.join(ROOT, "paper_2107_12720_gb300")


def _build(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    if not os.path.exists(os.path.join(LIBDIR, "libtrim.so")):
        pytest.skip("libtrim.so not built")
    exe = os.path.join(tmp_path, "trim_c_client")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           SRC, "-L", LIBDIR, "-ltrim", "-Wl,-rpath," + LIBDIR, "-o", exe])
    return exe


def test_c_client_without_device(tmp_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    exe = _build(tmp_path)
    r = subprocess.run([exe, "--expect-no-device"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.gpu
def test_c_client_on_device(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and "c client ok" in r.stdout, r.stdout + r.stderr
