"""The plane-window scheduling shared by the window gridding and degridding
(grid_win.cuh), checked on the host with the kernels' own helpers
(tests/csrc/grid_win_sched_check.cu, compiled by nvcc for the host and run
here; no GPU): the part split of a heavy tile covers each window's slots
once, the interleaved chunk walk visits every slot of every window exactly
once in window order with at most C slots a chunk, and the degridding's
clamped tap block holds exactly the footprint cells inside the tile."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
def test_window_schedule_and_tap_block(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "grid_win_sched_check"
    src = os.path.join(ROOT, "tests", "csrc", "grid_win_sched_check.cu")
    csrc = os.path.join(ROOT, "paper_2406_01342_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", csrc, "-I", os.path.join(ROOT, "include"), src, "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
