"""bench.py's host-side arithmetic on CPU: the roofline record of each kernel (algorithmic
bytes, or warp instructions issued, over the measured time, against the peak), the PCI ids
that pick the benchmarked GPU's clock samples, and the clock record itself."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6000.0}


def test_smooth_roofline_counts_read_and_write():
    nvox = 512 * 512 * 1024
    r = bench.kernel_roofline("smooth", 1.0, nvox, {}, PEAKS, 2000.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["algorithmic_bytes"] == 8 * nvox
    assert r["achieved"] == pytest.approx(8 * nvox / 1e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0, rel=1e-3)
    # beside it, what the three 1-D passes as separate sweeps would have to move in that time
    assert r["three_pass_bytes"] == 24 * nvox and r["three_pass_equiv_frac"] == pytest.approx(3 * r["frac"], rel=1e-3)
    # the zip form: the method's 8 bytes per voxel, and beside them the 16 it moves (it also
    # re-reads the first cube's result and writes the 8-byte pair)
    z = bench.kernel_roofline("smooth2", 1.0, nvox, {}, PEAKS, 2000.0)
    assert z["algorithmic_bytes"] == 8 * nvox and z["moved_bytes"] == 16 * nvox
    assert z["frac_moved"] == pytest.approx(2 * z["frac"], rel=1e-3)


def test_render_roofline_is_instruction_issue(monkeypatch):
    samples = {"mip": 10 ** 9, "composite": 10 ** 9, "ratio": 10 ** 9}
    monkeypatch.setattr(bench, "WARP_INST_PER_SAMPLE", {"mip": 3.5, "composite": 4.5, "ratio": 4.0})
    r = bench.kernel_roofline("render_mip", 2.0, 1, samples, PEAKS, 2000.0)
    peak = 152 * 4 * 2000e6 / 1e9  # warp instructions per second, in G
    assert r["bound"] == "alu" and r["unit"] == "Gwarp-inst/s" and r["peak"] == pytest.approx(peak, rel=1e-3)
    assert r["achieved"] == pytest.approx(3.5 * 1e9 / 2e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / peak, rel=1e-3)
    assert r["gsamples_per_s"] == pytest.approx(500.0)
    # beside it, the FP32 fraction of the method's flops
    fp32 = 152 * 128 * 2 * 2000e6 / 1e12
    assert r["fp32_frac_alg_flops"] == pytest.approx(bench.ALG_FLOPS_PER_SAMPLE["mip"] * 1e9 / 2e-3 / 1e12 / fp32,
                                                    rel=1e-3)
    # HBM fraction: the cube once (both cubes for the ratio) plus the image
    h = bench.kernel_roofline("render_ratio", 2.0, 10 ** 9, samples, PEAKS, 2000.0, image_bytes=160)
    assert h["algorithmic_bytes"] == 8 * 10 ** 9 + 160
    assert h["hbm_frac"] == pytest.approx((8e9 + 160) / 2e-3 / 1e9 / 6000.0, rel=1e-3)


def test_render_roofline_without_a_count_falls_back_to_flops(monkeypatch):
    samples = {"mip": 10 ** 9, "composite": 10 ** 9}
    monkeypatch.setattr(bench, "WARP_INST_PER_SAMPLE", {})
    r = bench.kernel_roofline("render_mip", 2.0, 1, samples, PEAKS, 2000.0)
    peak = 152 * 128 * 2 * 2000e6 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] == pytest.approx(peak, rel=1e-3)
    assert r["achieved"] == pytest.approx(bench.ALG_FLOPS_PER_SAMPLE["mip"] * 1e9 / 2e-3 / 1e12, rel=1e-3)
    c = bench.kernel_roofline("render_composite", 2.0, 1, samples, PEAKS, 2000.0)
    assert c["achieved"] > r["achieved"]  # compositing does the most per sample


def test_pci_key_ignores_domain_width_and_case():
    k = bench._pci_key
    assert k("00000008:01:00.0") == k("0008:01:00.0") == k("0008:01:00.0 ")
    assert k("0000:0A:00.0") == k("0000:0a:00.0")
    assert k("0009:01:00.0") != k("0008:01:00.0")
    assert k("not-a-bus-id") == "not-a-bus-id"


def test_clock_record_keeps_this_gpus_rows():
    cs = bench.ClockSampler(bus_id="0000:00:07.0")
    cs.lines = [
        "0, 00000000:00:07.0, 1980, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Active",
        "1, 00000000:00:08.0, 1200, 2070, 300.0, 0x0, Active, Not Active, Not Active, Not Active",
        "0, 00000000:00:07.0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    r = cs.summary()
    assert r["samples"] == 2 and r["sm_mhz"] == pytest.approx(2025.0) and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["gpu_pci"] == "0000:00:07.0"
    other = bench.ClockSampler(bus_id="0000:00:09.0")
    other.lines = cs.lines
    r2 = other.summary()
    assert r2["samples"] == 3 and r2["gpu_pci"] == "all listed GPUs"


def test_best_by_brick_edge_compares_unrounded_times():
    """The per-edge summary of a tuned plan picks what the autotuner picks: the smallest
    measured time (not a rounded one), the earlier candidate on a tie."""
    import bench
    cands = [(16, 2, 16, 50.0), (8, 8, 16, 43.07440), (8, 32, 16, 43.07420), (8, 16, 16, 43.07420),
             (16, 4, 32, 44.0), (8, 32, 32, 43.3461)]
    got = bench.best_by_brick_edge(cands)
    assert got == {"16": {"tile": 8, "ctas_per_sm": 32, "tune_ms": 43.074},
                   "32": {"tile": 8, "ctas_per_sm": 32, "tune_ms": 43.346}}
    assert bench.best_by_brick_edge([]) == {}
