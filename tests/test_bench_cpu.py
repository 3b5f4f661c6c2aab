"""Host logic of the measurement script (no GPU): the algorithmic work counts
behind the roofline objects against brute force, the roofline arithmetic on a
made-up kernel-class record, and the traffic record's source-hash check."""
import hashlib
import os
import types

import pytest

import bench


def _brute_gram_entries(n_new, n_act):
    # rows: the first n_new atoms; columns: all n_act atoms and V (index n_act);
    # a pair of new atoms is one entry (symmetry)
    seen = set()
    for r in range(n_new):
        for c in range(n_act + 1):
            seen.add((min(r, c), max(r, c)) if c < n_new else (r, c))
    return len(seen)


@pytest.mark.parametrize("n_new,n_act", [(1, 1), (1, 10), (5, 5), (16, 40), (873, 873)])
def test_gram_entries_is_the_distinct_count(n_new, n_act):
    assert bench.gram_entries(n_new, n_act) == _brute_gram_entries(n_new, n_act)


def test_tensor_core_iterations_and_phase_bytes():
    hist = [{"n_new": 873, "n_active": 873}, {"n_new": 1, "n_active": 177},
            {"n_new": 15, "n_active": 300}, {"n_new": 16, "n_active": 255},
            {"n_new": 16, "n_active": 256}, {"n_new": 0, "n_active": 19}]
    tc = bench.tc_iterations(hist)
    # the library's switch: at least 16 new atoms and n_new * n_active >= 4096
    assert tc == [hist[0], hist[4]]
    M = 1000
    # rows = active atoms + V, padded to 256; FP16 hi + lo of cos and sin = 8 B
    assert bench.phase_gen_bytes(M, hist) == 8.0 * M * (1024 + 512)


def test_roofline_arithmetic():
    wl = types.SimpleNamespace(M=200_000, N=512)
    info = {"grid_side": 1024, "n_planes": 8, "kernel_width": 7}
    hist = [{"n_new": 873, "n_active": 873, "n_support": 176, "apgd_iterations": 18}]
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0}
    steps = 5
    prof = {"gram_tc": (steps, steps, 5 * 0.9), "phase_gen": (steps, steps, 5 * 0.3),
            "grid": (35, 70, 35 * 0.1)}
    r = bench.roofline(prof, info, wl, hist, steps, peaks, "gram_tc")
    flop = 12.0 * wl.M * bench.gram_entries(873, 873)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flop / 0.9e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 2000.0)
    p = bench.roofline(prof, info, wl, hist, steps, peaks, "phase_gen")
    assert p["bound"] == "hbm"
    assert p["achieved"] == pytest.approx(8.0 * wl.M * 1024 / 0.3e-3 / 1e9)
    g = bench.gridding_roofline(prof, info, wl, peaks)
    assert g["bytes_per_launch"] == 20.0 * wl.M + 8.0 * 8 * 1024 * 1024
    assert g["avg_launch_ms"] == pytest.approx(0.1)
    assert g["vis_per_s"] == pytest.approx(wl.M / 0.1e-3)
    # the spread's FP32 work: a complex value times a real weight (2 FMA) per
    # footprint cell, W^3 cells with w-stacking, W^2 without
    assert g["alu_flops_per_launch"] == 4.0 * wl.M * 7 ** 3
    assert g["alu_frac"] == pytest.approx(4.0 * wl.M * 343 / 0.1e-3 / 1e12 / (152 * 128 * 2 * 2.07e9 / 1e12))
    r = bench.roofline(prof, info, wl, hist, steps, peaks, "grid")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(g["alu_achieved_tflops"])
    assert bench.gridding_flops(wl.M, dict(info, n_planes=1)) == 4.0 * wl.M * 49
    # the degridding's interpolation: the spread's FMAs in reverse, per launch
    prof["degrid"] = (10, 20, 10 * 0.08)
    d = bench.roofline(prof, info, wl, hist, steps, peaks, "degrid")
    assert d["bound"] == "alu" and d["achieved"] == pytest.approx(4.0 * wl.M * 343 / 0.08e-3 / 1e12)
    # its FFT passes: image read, reachable grid written, pass-1 rows written and read
    prof["degrid_fft"] = (10, 20, 10 * 0.05)
    reach = {"rows": 512, "col_groups": 16}
    f = bench.roofline(prof, info, wl, hist, steps, peaks, "degrid_fft", reach)
    cells = 512 * 16 * 32
    assert f["bound"] == "hbm"
    assert f["achieved"] == pytest.approx((4.0 * 512 * 512 + 8.0 * 8 * cells + 16.0 * 8 * 512 * 512) / 0.05e-3 / 1e9)


def test_traffic_record_needs_the_profiled_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2406_01342_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "k.cu"
    src.write_bytes(b"kernel source v1\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "k.md").write_text(
        f"text\ntraffic-record: class=gram_tc bytes_per_launch=123 kernels=k sources=k.cu:{h}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("gram_tc") == 123.0
    assert bench.recorded_traffic("grid") is None
    src.write_bytes(b"kernel source v2\n")      # the kernel changed since the capture
    assert bench.recorded_traffic("gram_tc") is None
    os.remove(src)
    assert bench.recorded_traffic("gram_tc") is None


def test_cpu_baseline_runs_the_oracle_over_the_host_cores():
    """The CPU baseline leg: spawned one-thread oracle processes on every core
    this process may use, the CPU model named, the extrapolation labelled."""
    value, base = bench.oracle_solves_per_s("tiny_64_coplanar", 4, target_s=0.3)
    info = bench.host_cpu()
    assert value > 0 and base["value"] == value
    assert base["cores"] == info["cores"] >= 1 and base["nproc"] == info["cores"]
    assert isinstance(base["cpu_model"], str) and base["cpu_model"]
    assert base["extrapolated"] is True and "EXTRAPOLATED" in base["sample"]
    assert base["certificates"] == 4 and base["kind"] == "oracle"
