"""Host logic of bench.py behind the figures that qualify a measurement:
the clock record of the timed region (median SM clock, its maximum, and the
throttle reasons seen active; a number taken with hw_slowdown,
hw_thermal_slowdown or sw_thermal_slowdown active does not stand), the
roofline denominators (the measured peaks file, else the stated fallback),
and the replica figures of a single rank."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(dev, sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"{dev}, {sm}, {mx}, 812.50, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}\n"


def test_clock_summary_median_max_and_active_reasons(tmp_path):
    p = tmp_path / "clocks.csv"
    p.write_text("".join([
        _line(0, 2070, 2070),
        _line(0, 1995, 2070, cap="Active"),
        _line(1, 900, 2070, hw="Active"),          # another GPU: ignored
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n",   # unreadable: skipped
        _line(0, 2040, 2070),
        "garbage\n",
    ]))
    s = bench._clock_summary(str(p), 0)
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_every_slowdown_kind(tmp_path):
    p = tmp_path / "clocks.csv"
    p.write_text(_line(0, 1500, 2070, hw="Active") + _line(0, 1400, 2070, hwt="Active")
                 + _line(0, 1450, 2070, swt="Active"))
    s = bench._clock_summary(str(p), 0)
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1450.0


def test_clock_summary_without_a_record(tmp_path):
    s = bench._clock_summary(str(tmp_path / "missing.csv"), 0)
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_peaks_come_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench._load_peaks()
    assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7100.0, "bf16_tflops": 2000.0}))
    peaks, kind = bench._load_peaks()
    assert kind == "measured" and peaks["hbm_gbs"] == 7100.0


def test_replicas_of_one_rank_report_the_rank_itself():
    ms, units, rate = bench.replica_throughput(None, 4.0, 1000)
    assert (ms, units) == (4.0, 1000.0) and rate == 250_000.0


def test_reference_arm_names_its_modes():
    """The reference arm times the oracle for the grad and cycle modes only;
    any other mode gets the unavailable line instead of another mode's figure."""
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--mode", "edm"],
                         capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-500:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "grad" in line["unavailable"]
