"""Host-side helpers of bench.py: the HBM roofline figures and the gate on committed traffic."""
import hashlib
import os

import pytest

import bench


def test_algorithmic_bytes_per_cell_match_the_method():
    # no bulk h between iterations (Sec. 3.1): code byte + (d + 1) FP64 moments read +
    # 2^d (d + 1) FP32 partials written; per update 73 / 1024 (2D, 32^2 velocities) and
    # 161 / 4096 (3D, 16^3 velocities)
    h2 = bench.hbm_fractions({"hbm_gbs": 1000.0}, 2, 10, 1e-3, 1e-3, None)
    h3 = bench.hbm_fractions({"hbm_gbs": 1000.0}, 3, 10, 1e-3, 1e-3, None)
    assert h2["algorithmic_bytes_per_cell"] == 73
    assert h3["algorithmic_bytes_per_cell"] == 161
    assert 73 / 1024 == pytest.approx(0.0713, abs=1e-4)
    assert 161 / 4096 == pytest.approx(0.0393, abs=1e-4)
    assert h2["dram_gbs"] is None and h2["dram_frac"] is None


def test_hbm_fractions_divide_by_the_right_times():
    peaks = {"hbm_gbs": 5000.0}
    cells = 1 << 20
    h = bench.hbm_fractions(peaks, 3, cells, sweep_s=2e-3, iter_s=4e-3, traffic=10_000_000_000)
    assert h["peak_gbs"] == 5000.0 and "measured" in h["peak_basis"]
    assert h["algorithmic_bytes_per_iteration"] == 161 * cells
    # algorithmic bytes over the whole iteration's time, measured bytes over the sweep's
    assert h["algorithmic_gbs"] == pytest.approx(161 * cells / 4e-3 / 1e9, abs=0.1)
    assert h["dram_gbs"] == pytest.approx(5000.0)
    assert h["dram_frac"] == pytest.approx(1.0)


def test_hbm_fallback_peak_is_named():
    h = bench.hbm_fractions({}, 2, 100, 1e-3, 1e-3, None)
    assert h["peak_gbs"] == bench.HBM_FALLBACK_GBS and "fallback" in h["peak_basis"]


def _fake_tree(tmp_path, body):
    src = tmp_path / "k.cu"
    src.write_text(body)
    (tmp_path / "profiles").mkdir()
    digest = hashlib.sha256(body.encode()).hexdigest()
    (tmp_path / "profiles" / "p.md").write_text(
        "text\n```\ntraffic_kernel: k<8>\ntraffic_tiles: 8 4 4\n"
        "traffic_source_sha256: %s\ntraffic_bytes_per_launch: 12345\n```\n" % digest)
    return src


def test_measured_traffic_needs_same_sources_and_tiles(tmp_path, monkeypatch):
    src = _fake_tree(tmp_path, "kernel source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_PROFILES", {"w": ("p.md", ("k.cu",))})
    assert bench.measured_traffic("w", (8, 4, 4)) == 12345
    assert bench.measured_traffic("w", (8, 4, 8)) is None          # another tile shape
    assert bench.measured_traffic("other", (8, 4, 4)) is None      # no capture of that workload
    src.write_text("kernel source, edited\n")
    assert bench.measured_traffic("w", (8, 4, 4)) is None          # sources changed since the capture


def test_committed_traffic_profiles_parse():
    # every committed traffic block names its kernel, tiles, source hash and a byte count
    for workload, (fname, sources) in bench.TRAFFIC_PROFILES.items():
        text = open(os.path.join(bench.ROOT, "profiles", fname)).read()
        fields = dict(l.split(": ", 1) for l in text.splitlines() if l.startswith("traffic_"))
        assert set(fields) >= {"traffic_kernel", "traffic_tiles", "traffic_source_sha256",
                               "traffic_bytes_per_launch"}, workload
        assert int(fields["traffic_bytes_per_launch"]) > 0
        assert len(fields["traffic_source_sha256"]) == 64
        for f in sources:
            assert os.path.exists(os.path.join(bench.ROOT, f))


_SMI = [
    "0, 2070, 2070, 812.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 2055, 2070, 1302.11, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2070, 2070, 1390.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 345, 2070, 110.20, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active",
    "[N/A], [N/A]",
    "0, [N/A], 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
]


def test_parse_clocks_takes_the_median_under_load_and_every_active_reason():
    c = bench.parse_clocks(_SMI)
    assert c["samples"] == 4                       # malformed and N/A lines are skipped
    assert c["sm_max_mhz"] == 2070.0
    assert c["sm_mhz"] == 2070.0                   # median of 2070, 2055, 2070 (345 MHz idle sample left out)
    assert c["reasons"] == ["sw_power_cap"]
    hot = _SMI[0].replace("Not Active, Not Active, Not Active, Not Active",
                          "Active, Active, Not Active, Not Active")
    assert bench.parse_clocks([hot])["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert bench.parse_clocks([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_clock_sampler_stop_parses_its_file(tmp_path):
    import subprocess
    s = bench.ClockSampler(0, str(tmp_path))
    with open(s.path, "w") as f:
        f.write("\n".join(_SMI) + "\n")
    s.fh = open(os.devnull, "w")
    s.proc = subprocess.Popen(["sleep", "30"])    # stands in for the sampling process
    c = s.stop()
    assert s.proc.poll() is not None
    assert c["samples"] == 4 and c["sm_mhz"] == 2070.0 and c["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi_says_so(tmp_path):
    s = bench.ClockSampler(0, str(tmp_path))
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
