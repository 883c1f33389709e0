"""The benchmark's measurement helpers, on the CPU: the clock record taken
during the timed region (median SM clock under load, throttle reasons seen
under load), the committed ncu figures (used only while the profiled
kernel's sources are unchanged), the issue-rate entry and the per-kernel
share table."""
import hashlib
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _DoneProc:
    """Stands in for the finished nvidia-smi process."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _line(sm, smax, util, hw="Not Active", thermal="Not Active", swthermal="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, 900.5, 0x0, {hw}, {thermal}, {swthermal}, {cap}, {util}"


def _stop(lines):
    s = bench.ClockSampler("0")
    s.proc = _DoneProc()
    s.lines = list(lines)
    return s.stop()


def test_clock_record_takes_loaded_samples_only():
    rec = _stop([
        _line(345, 2070, 0, cap="Active"),  # idle sample: its clock and reasons are not the timed region's
        _line(2070, 2070, 97),
        _line(2055, 2070, 100, cap="Active"),
        _line(2070, 2070, 88),
        "garbage line",
        _line("[N/A]", 2070, 90),  # unreadable clock: skipped
    ])
    assert rec["sm_mhz"] == 2070.0  # median of 2070, 2055, 2070
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert rec["samples_under_load"] == 3 and rec["samples"] == 6


def test_clock_record_reports_every_slowdown_seen_under_load():
    rec = _stop([_line(1600, 2070, 100, hw="Active"), _line(1500, 2070, 100, thermal="Active", swthermal="Active")])
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert rec["sm_mhz"] == 1550.0


def test_clock_record_without_nvidia_smi():
    s = bench.ClockSampler("0")
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}


@pytest.fixture()
def fake_root(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({
        "k_case": {"bytes_per_launch": 1234, "inst_per_launch": 4.0e6, "sources": {"k.cu": h}},
        "k_noinst": {"bytes_per_launch": 99, "sources": {"k.cu": h}},
    }))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return src


def test_profile_figures_hold_only_while_sources_are_unchanged(fake_root):
    assert bench.traffic_from_profile("k_case") == 1234.0
    assert bench.traffic_from_profile("missing") is None
    fake_root.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.profile_record("k_case") is None
    assert bench.traffic_from_profile("k_case") is None
    assert bench.issue_from_profile("k_case", 0.01, {"sm_mhz": 2000.0}, 152) is None


def test_issue_rate_arithmetic(fake_root):
    got = bench.issue_from_profile("k_case", 0.005, {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0}, 152)
    # 4e6 warp instructions in 5 us against 152 SMs x 4 schedulers x 2.0 GHz
    assert got["achieved_per_s"] == pytest.approx(8.0e11)
    assert got["peak_per_s"] == pytest.approx(1.216e12)
    assert got["frac"] == pytest.approx(8.0e11 / 1.216e12, abs=1e-4)
    # the maximum clock stands in when no loaded sample was taken
    alt = bench.issue_from_profile("k_case", 0.005, {"sm_mhz": None, "sm_max_mhz": 2070.0}, 152)
    assert alt["peak_per_s"] == pytest.approx(4 * 152 * 2070e6)
    assert bench.issue_from_profile("k_case", 0.005, {}, 152) is None
    assert bench.issue_from_profile("k_case", 0.0, {"sm_mhz": 2000.0}, 152) is None
    assert bench.issue_from_profile("k_noinst", 0.005, {"sm_mhz": 2000.0}, 152) is None


def test_kernel_table_shares():
    steps = [[("a", 1.0), ("b", 0.5), ("b", 0.5)], [("a", 3.0), ("b", 1.0), ("b", 1.0)]]
    t = bench.kernel_table(steps)
    assert list(t) == ["a", "b"]  # by total time
    assert t["a"] == {"launches_per_step": 1, "ms_per_launch": 2.0, "share": round(4.0 / 7.0, 4)}
    assert t["b"]["launches_per_step"] == 2 and t["b"]["ms_per_launch"] == 0.75
    assert t["a"]["share"] + t["b"]["share"] == pytest.approx(1.0, abs=1e-4)
    assert bench.kernel_table([]) == {}


def test_committed_profile_records_are_well_formed():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        prof = json.load(f)
    assert prof
    for key, ent in prof.items():
        assert ent["bytes_per_launch"] > 0, key
        assert os.path.isfile(os.path.join(ROOT, ent["profile"])), key
        for src, h in ent["sources"].items():
            assert os.path.isfile(os.path.join(ROOT, src)), (key, src)
            assert len(h) == 16 and int(h, 16) >= 0
