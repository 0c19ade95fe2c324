"""Host logic of bench.py on the CPU: the clock summary that decides whether a
timed run is kept (median SM clock under load, throttle reasons seen), the
HBM peak lookup, the whole-job value and the reference arm's JSON line.  No
GPU, no nvidia-smi."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _row(sm, mx, hw="Not Active", therm="Not Active", swth="Not Active", cap="Not Active"):
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, therm, swth, cap]


def test_clock_summary_median_and_reasons():
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.rows = [_row(2070, 2070), _row(2070, 2070, cap="Active"), _row(1980, 2070), ["garbage"],
              _row("[N/A]", 2070)]
    out = c.stop()
    assert out["sm_mhz"] == 2070.0  # median of 2070, 2070, 1980
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 5


def test_clock_summary_flags_thermal_slowdown():
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.rows = [_row(1500, 2070, therm="Active"), _row(1400, 2070, hw="Active")]
    out = c.stop()
    assert set(out["reasons"]) == {"hw_slowdown", "hw_thermal_slowdown"}


def test_clock_summary_without_nvidia_smi():
    c = bench.ClockSampler(0)
    out = c.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_peaks_reads_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.FALLBACK_HBM, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6783.5}))
    assert bench.peaks() == (6783.5, "measured")


def test_job_value_counts_all_replicas():
    assert bench.job_value(1, 500, 1, 40000.0) == pytest.approx(12.5)
    assert bench.job_value(4, 500, 2, 80000.0) == pytest.approx(50.0)


def test_reference_arm_prints_one_complete_line():
    """The reference arm (the CPU oracle on its bounded sample) runs without a
    GPU and prints one JSON line with the keys the bench contract asks for."""
    import subprocess

    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "leftmost eigenpairs/sec to residual 1e-8" and d["unit"] == "eigenpairs/s"
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["config"]["workload"] == bench.WORKLOAD["workload"]
    assert d["config"]["sample"]["npts"] == bench.SAMPLE["npts"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
