"""Host-side pins of the polyphase order and the z layout of the framelet
kernels (no GPU): tests/host/layout_check.cu includes the library's own
header, is compiled by nvcc as host code and run here."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else None


def test_polyphase_order_and_z_layout(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "layout_check")
    src = os.path.join(HERE, "host", "layout_check.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-o", exe, src], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
