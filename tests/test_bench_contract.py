"""bench.py's output contract: one JSON line with the keys the benchmark driver reads.

The reference arm (the CPU oracle on the host cores) runs here on the CPU; the default arm
needs a GPU and runs a short version of the benchmark step."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=timeout, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--steps", "3", "--warmup", "3"], timeout=600)
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "Gpoint-updates/s" and d["higher_is_better"] is True
    assert d["steps"] == 3 and d["warmup"] == 3 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"] == bench.workload_config(256, 1)


@pytest.mark.gpu
def test_default_arm_line():
    d = _run(["--steps", "5", "--warmup", "3", "--no-cpu-baseline", "--no-stencil", "--no-plain"], timeout=900)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["n_gpus"] == 1 and d["steps"] == 5 and d["warmup"] == 3 and d["dtype"] == "f64"
    assert d["config"] == bench.workload_config(256, 1) and d["form"] == "saturated"
    r = d["roofline"]
    assert r["bound"] == "alu" and 0 < r["frac"] <= 1.05 and r["achieved"] == pytest.approx(r["frac"] * r["peak"])
    assert d["gpu_launches"] == 5
    # the roofline's peak is the FP64 probe measured in the run; the derived peak sits beside it
    assert r["peak"] == pytest.approx(d["fp64_probe"]["gops"]) and r["peak_derived"] > 0
    assert 1.5 < d["fp64_probe"]["op_per_clk_per_sm"] <= 2.05
    # in-process clock samples over the timed legs
    assert d["clocks"]["samples"] >= 10 and d["clocks"]["sm_mhz"] > 0
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == 703040000 and e["d2h_bytes_per_step"] == 671088640
    # the host link measured under the step: moving both directions at once is its floor
    link = e["host_link"]
    assert 0 < link["both_ms"] <= e["ms_per_step"] * 1.02
    assert link["upload_gbs"] > 50 and link["download_gbs"] > 50


class _FakeNvml:
    """Stands in for the NVML wrapper: fixed readings, counts the queries."""

    def __init__(self):
        self.calls = 0

    def sm_mhz(self):
        self.calls += 1
        return 2070.0

    def power_w(self):
        return 300.0

    def reasons(self):
        return []


def test_clock_sampler_windows_and_pause():
    """The sampler keeps only samples inside registered windows, and queries nothing while paused."""
    import time
    sm = bench.ClockSampler(0, period_s=0.002)
    sm.nvml, sm.max_mhz = _FakeNvml(), 2070.0
    sm.start()
    time.sleep(0.05)
    sm.pause()
    time.sleep(0.01)              # a query already under way may still land
    n0 = sm.nvml.calls
    time.sleep(0.05)
    assert sm.nvml.calls == n0    # no queries while paused
    sm.resume()
    t0 = time.time()
    time.sleep(0.05)
    t1 = time.time()
    sm.window(t0, t1)
    sm.stop()
    s = sm.summary()
    assert s["samples"] >= 5 and s["sm_mhz"] == 2070.0 and s["reasons"] == []
    assert all(t0 <= r[0] <= t1 for r in sm.samples if t0 <= r[0] <= t1)
    assert s["samples"] < len(sm.samples)   # samples outside the window are not counted


def test_workload_config_is_shared_by_both_arms():
    c = bench.workload_config(256, 1)
    assert c["workload"] == "rhs_256^3_fp64" and c["grid"] == [256] * 3 and c["h"] == [1.0, 1.0, 1.0]
    assert "703 MB in, 671 MB out" in c["l2"] and c["parallelism"] == "replicas x1"
