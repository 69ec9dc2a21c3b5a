"""Host-side checks of the kernel-pool and node-vector layouts (no GPU needed).

The FP32 sweeps stream a row group's kernel entries over any column range as one bulk copy and
read them as float4 from shared memory; these properties of kpos / vpos (csrc/qdse_internal.h) are
what that relies on: both maps are one-to-one, every 4-aligned column range of a group is one
contiguous run starting where the sweep computes it, a block's 4 columns are adjacent, and the
swizzle of full groups spreads a quarter warp's 16-byte reads over 8 bank quads.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_pool_and_vector_layouts(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "check_layout")
    src = os.path.join(HERE, "layout", "check_layout.cu")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-o", exe, src], check=True,
                   capture_output=True, timeout=300)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout + out.stderr
