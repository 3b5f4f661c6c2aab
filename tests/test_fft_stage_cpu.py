"""The one-CTA FFT's shared-memory staging map (fft_cta.cuh: stage_mask /
stage_pos, the swizzle that keeps the staged outputs of the row passes free
of bank conflicts) is checked on the host with the kernels' own lane
mappings: a bijection inside every group of R slots, one mask per lane, and
16 different eight-byte bank pairs for every half-warp store and every
aligned read-back run (tests/csrc/fft_stage_check.cu, compiled by nvcc for
the host and run here; no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
def test_fft_staging_swizzle_is_a_conflict_free_bijection(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "fft_stage_check"
    src = os.path.join(ROOT, "tests", "csrc", "fft_stage_check.cu")
    csrc = os.path.join(ROOT, "paper_2406_01342_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", csrc, "-I", os.path.join(ROOT, "include"), src, "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
