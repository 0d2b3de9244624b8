"""bench.py's host-side helpers (CPU): the clock summary that decides whether
a run is kept, and the traffic record keyed to the kernel source."""
import json
import os

import bench


OK_LINE = "0, {sm}, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, {cap}"


def test_clock_summary_median_max_and_throttle_reasons():
    s = bench.ClockSampler(0)
    lines = [OK_LINE.format(sm=m, cap="Not Active") for m in (2070, 2055, 2040)]
    lines += [OK_LINE.format(sm=1980, cap="Active"), "garbage", "0, [N/A], 2070, 1, 0, a, b, c, d"]
    s.lines = [(float(k), ln) for k, ln in enumerate(lines)]
    out = s.summary()
    assert out["sm_mhz"] == 2047.5 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 4
    # only the samples that arrived inside the timed window count
    s.mark(0.5, 2.0)
    out = s.summary()
    assert out["samples"] == 2 and out["sm_mhz"] == 2047.5 and out["reasons"] == []
    hot = "0, 1500, 2070, 1300, 0x48, Not Active, Active, Not Active, Not Active"
    s.lines, s.window = [(0.0, hot)], None
    assert s.summary()["reasons"] == ["hw_thermal_slowdown"]
    s.lines = []
    assert s.summary()["sm_mhz"] is None


def test_clock_sampler_runs_nvidia_smi_through_the_timed_window(tmp_path, monkeypatch):
    """A stand-in nvidia-smi on PATH prints a sample every 50 ms; the sampler
    waits for the first one, and the window keeps the samples taken in it."""
    import sys
    import time
    fake = tmp_path / "nvidia-smi"
    script = ["#!" + sys.executable, "import time", "for k in range(200):",
              "    print(%r.format(sm=2000 + k %% 7, cap='Not Active'), flush=True)" % OK_LINE,
              "    time.sleep(0.05)"]
    fake.write_text("\n".join(script) + "\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    with bench.ClockSampler(0) as clk:
        assert clk.lines                                  # sampling started before the window
        t0 = time.monotonic()
        time.sleep(0.5)
        clk.mark(t0, time.monotonic())
    out = clk.summary()
    assert 5 <= out["samples"] <= 15
    assert 2000 <= out["sm_mhz"] <= 2006 and out["reasons"] == []


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    with bench.ClockSampler(0) as clk:
        clk.mark(0.0, 1.0)
    assert clk.summary()["sm_mhz"] is None


def test_traffic_record_only_for_the_current_kernel_source(tmp_path, monkeypatch):
    root = tmp_path
    (root / "profiles").mkdir()
    (root / "paper_2208_12335_gb300" / "csrc").mkdir(parents=True)
    src = root / "paper_2208_12335_gb300" / "csrc" / "k.cu"
    src.write_bytes(b"kernel source v1\n")
    import hashlib
    h = hashlib.sha256(b"kernel source v1\n").hexdigest()[:16]
    rec = {"h": {"source": "k.cu", "source_sha256_16": h, "dram_bytes_per_algorithmic_flop": 0.125,
                 "workload": "chno1000"}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_for("h") == 0.125
    assert bench.traffic_for("density") is None
    assert bench.traffic_for("h", "si64") is None              # taken on another workload
    src.write_bytes(b"kernel source v2\n")                 # the kernel changed since the capture
    assert bench.traffic_for("h") is None


def test_measured_peaks_file_is_read():
    peaks, kind = bench.measured_peaks()
    assert kind in ("measured", "fallback")
    assert peaks["hbm_gbs"] > 0 and peaks["bf16_tflops"] > 0
