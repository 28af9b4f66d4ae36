"""Host logic of the merged-order tiling and the batch layout (csrc/layout.h),
compiled as a small host program: tie order, tile limits, per-marginal counts,
the threaded merge above a million points against a plain sort, the padded
stream of the tile kernels,
instance offsets and zero decays across instance boundaries."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return os.path.join(c, "include")
    return None


def test_layout_host(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("g++ or CUDA headers not available")
    exe = str(tmp_path / "layout_check")
    src = os.path.join(ROOT, "tests", "host", "layout_check.cpp")
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I" + inc,
                    "-I" + os.path.join(ROOT, "paper_2405_19246_gb300", "csrc"),
                    "-I" + os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
