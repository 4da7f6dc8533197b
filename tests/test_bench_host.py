"""bench.py's host-side legs on CPU: the reference arm's JSON line (the CPU
oracle as the reference implementation), the CPU baseline record (all cores
and one core), and the recorded-traffic lookup."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "Gpixel/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    # the same config dict as our arm prints, so the two lines compare
    assert line["config"] == bench.workload_config(1)
    assert len(line["input_sha256"]) == 64


def test_cpu_baseline_record_has_all_core_and_one_core_rates():
    img = synth.rects_noise(300, 512, 1)
    rec = bench.cpu_baseline(img, 0.3)
    assert rec["kind"] == "oracle" and rec["unit"] == "Gpixel/s"
    assert rec["value"] > 0 and rec["cores"] >= 1
    assert rec["one_core"]["value"] > 0 and "1 thread" in rec["one_core"]["sample"]


def test_recorded_traffic_is_bytes_or_none():
    t = bench.recorded_traffic("tma")
    assert t is None or (isinstance(t, int) and t > 5 * 8192 * 8192 // 2)
    assert bench.recorded_traffic("no_such_kernel") is None
    for stem in ("tma", "lanecopy", "tc"):
        assert len(bench.kernel_source_hash(stem)) == 16
    assert bench.kernel_source_hash("tma") != bench.kernel_source_hash("tc")
    assert np.isfinite(bench.weak_scaling_value(100, 2, 1, 1.0))
