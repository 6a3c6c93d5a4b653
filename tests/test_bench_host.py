"""Host logic of bench.py that decides what the benchmark line reports, on
the CPU: the clock record taken from nvidia-smi samples during the timed
region (median SM clock, highest maximum clock, every throttle reason seen
active) and the peaks read from the measured-peaks file."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeSampler:
    """Stands in for the nvidia-smi process: already finished."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _clocks_from(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(ln + "\n" for ln in lines))
    c = bench.Clocks(0)
    c.proc = _FakeSampler()
    c.path = str(path)
    c.f = open(os.devnull, "w")
    return c.stop()


def test_clock_record_from_samples(tmp_path):
    lines = [
        "0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    rec = _clocks_from(tmp_path, lines)
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2055.0                      # median of 2070, 2040, 2055
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(tmp_path / "clocks.csv")


def test_clock_record_names_every_slowdown(tmp_path):
    lines = ["0, 1500, 2070, 1400, 0x68, Active, Active, Active, Not Active",
             "0, 1600, 2070, 1400, 0x0, Not Active, Not Active, Not Active, Not Active"]
    rec = _clocks_from(tmp_path, lines)
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert rec["sm_mhz"] == 1550.0


def test_no_sampler_gives_an_empty_record():
    c = bench.Clocks(0)
    assert c.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_measured_peak_reads_the_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak("hbm_gbs", 6800.0) == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6674.5}))
    assert bench.measured_peak("hbm_gbs", 6800.0) == 6674.5
    assert bench.measured_peak("bf16_tflops", 1900.0) == 1900.0
