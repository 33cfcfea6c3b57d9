"""Host helpers of bench.py: which step kernel a tile variant launches and how
many launches a step takes, the DRAM bytes read from a profile summary only
when its kernel-source hash is the current one, and the peak's fallback."""
import json
from types import SimpleNamespace

import bench


def test_kernel_name_and_launch_count():
    assert bench.kernel_name((52, 28, 512)) == "k_step_batch"
    assert bench.kernel_name((0, 48, 0)) == "k_march_batch"
    assert bench.kernel_name((64, 16, 256), bench.KIND_SPLIT, 0) == "k_flow_batch+k_energy_batch"
    assert bench.kernel_name((64, 16, 256), bench.KIND_SPLIT, 96) == "k_flow_batch+k_energy_walk_batch"
    assert bench.variant_key((64, 16, 256), bench.KIND_SPLIT, 96) == "64x16x256_walk96"
    assert bench.variant_key((64, 16, 256), bench.KIND_SPLIT, 0) == "64x16x256_tile"
    assert bench.variant_key((52, 28, 512)) == "52x28x512"
    assert bench.profile_name((64, 16, 256), bench.KIND_SPLIT) == "k_flow_energy_batch"
    cases = [SimpleNamespace(nx=n) for n in (256, 320, 300, 512, 500)]
    assert bench.step_launches(cases, (52, 20, 512)) == 1
    # row strides 256, 320 (300 rounds up to 320), 512 (500 too)
    assert bench.step_launches(cases, (0, 32, 0), bench.KIND_MARCH) == 3
    # a flow launch and one energy launch per sub-step of Eq. (27)
    assert bench.step_launches(cases, (64, 16, 256), bench.KIND_SPLIT) == 2
    assert bench.step_launches(cases, (64, 16, 256), bench.KIND_SPLIT, nsub=3) == 4


def _profile(root, h, lines, name="k_step_batch"):
    (root / "profiles").mkdir(parents=True, exist_ok=True)
    body = ["# summary", f"- kernel_source_hash: `{h}`"] + lines
    (root / "profiles" / f"{name}_sweep32.md").write_text("\n".join(body) + "\n")


def test_traffic_is_read_only_for_the_current_kernel(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc123")
    assert bench.read_traffic((52, 28, 512)) is None  # no summary
    _profile(tmp_path, "abc123", ["- dram_bytes_per_launch_full_sweep_52x28x512: 351090176",
                                  "- dram_bytes_per_launch_full_sweep_52x20x512: not-a-number"])
    assert bench.read_traffic((52, 28, 512)) == 351090176.0
    assert bench.read_traffic((52, 20, 512)) is None      # unparsable
    assert bench.read_traffic((52, 16, 256)) is None      # not captured
    _profile(tmp_path, "stale0", ["- dram_bytes_per_launch_full_sweep_52x28x512: 351090176"])
    assert bench.read_traffic((52, 28, 512)) is None      # kernel changed since the capture
    # split variants: one summary for the split step, keyed by the energy kernel
    _profile(tmp_path, "abc123", ["- dram_bytes_per_launch_full_sweep_64x16x256_walk96: 476000000"],
             name="k_flow_energy_batch")
    assert bench.read_traffic((64, 16, 256), bench.KIND_SPLIT, 96) == 476000000.0
    assert bench.read_traffic((64, 16, 256), bench.KIND_SPLIT, 64) is None
    assert bench.read_traffic((64, 16, 256), bench.KIND_SPLIT, 0) is None


def test_peak_prefers_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peak_gbs() == (6800.0, "of fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6789.3}))
    assert bench.peak_gbs() == (6789.3, "of measured")


def test_clock_samples_are_summarised():
    lines = ["2070, 2070, 812.5, Not Active, Not Active, Not Active, Not Active",
             "1995, 2070, 1390.1, Not Active, Not Active, Not Active, Active",
             "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active",
             "short line",
             "2040, 2070, 1201.0, Not Active, Active, Not Active, Not Active"]
    out = bench.parse_clock_lines(lines)
    assert out == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["hw_thermal_slowdown", "sw_power_cap"],
                   "samples": 3}
    assert bench.parse_clock_lines([])["sm_mhz"] is None
    # a malformed maximum-clock field keeps the sample's clock and its throttle reasons
    out = bench.parse_clock_lines(["1980, [N/A], 1000.0, Active, Not Active, Not Active, Not Active"])
    assert out["sm_mhz"] == 1980.0 and out["sm_max_mhz"] is None and out["reasons"] == ["hw_slowdown"]
