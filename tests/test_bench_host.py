"""Host-side pieces of bench.py that decide what a measurement reports, on the
CPU: the clock record parsed from nvidia-smi samples (median SM clock and the
throttle reasons that make a run invalid), the DRAM traffic figure that is
reported only for the kernel source it was measured on, and the peak figures
with their fallback."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s.summary()


def test_clock_summary_median_and_reasons():
    ok = "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1200.0, 0x0000000000000020, Not Active, Active, Not Active, Not Active"
    s = sampler([ok, ok, capped])
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    s = sampler([ok, hot, hot])
    assert s["sm_mhz"] == 1500.0 and s["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_skips_malformed_lines():
    s = sampler(["", "garbage", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active",
                 "0, 2000, 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert s["samples"] == 1 and s["sm_mhz"] == 2000.0 and s["reasons"] == []
    s = sampler([])
    assert s["sm_mhz"] is None and s["samples"] == 0


def test_traffic_reported_only_for_the_measured_kernel_source(tmp_path, monkeypatch):
    """The figure is used only while the kernel's source region hashes as
    when the counters were taken: an edit inside the region drops it, an
    edit outside does not."""
    import hashlib
    rel_src = os.path.join("paper_1602_06097_gb300", "csrc", "modgemm.cu")
    rel_prof = os.path.join("profiles", "dram_traffic_fl_150000x200000.md")
    os.makedirs(tmp_path / os.path.dirname(rel_src), exist_ok=True)
    os.makedirs(tmp_path / "profiles", exist_ok=True)
    shutil.copy(os.path.join(ROOT, rel_src), tmp_path / rel_src)
    code = open(tmp_path / rel_src).read()
    begin, end = "namespace tc {", "// Gathered product: the sparse operand compacted per column tile"
    a, b = code.index(begin), code.index(end)
    digest = hashlib.sha256(code[a:b].encode()).hexdigest()
    (tmp_path / rel_prof).write_text(f"traffic_bytes_per_launch: 739917251\n"
                                     f"launches_per_reduction: 268\n"
                                     f'kernel_region: modgemm.cu "{begin}" .. "{end}"\n'
                                     f"kernel_source_sha256: {digest}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic() == 739917251
    assert bench.profiled_traffic(launches=268.0) == 739917251
    assert bench.profiled_traffic(launches=340.0) is None       # another launch mix
    with open(tmp_path / rel_src, "a") as f:          # outside the region
        f.write("\n// edited\n")
    assert bench.profiled_traffic() == 739917251
    open(tmp_path / rel_src, "w").write(code[:a + 20] + "// edited\n" + code[a + 20:])   # inside
    assert bench.profiled_traffic() is None
    os.remove(tmp_path / rel_prof)
    assert bench.profiled_traffic() is None


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench.measured_peaks()
    assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6777.0, "bf16_tflops": 1936.2}')
    peaks, kind = bench.measured_peaks()
    assert kind == "measured" and peaks["hbm_gbs"] == 6777.0
