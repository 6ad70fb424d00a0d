"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the contract's keys, on a tiny sample (no GPU)."""
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--cpu-sample", "8"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    wall_ms = (time.perf_counter() - t0) * 1e3
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["metric"].startswith("image-samples/s") and d["unit"] == "image-samples/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "sample" in d["cpu_baseline"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] and d["config"]["images"] == 92168
    # the step time is what was timed (the bounded sample), so the timed steps
    # fit in the run; the full-scene extrapolation has its own key
    assert 0 < d["ms_per_step"] * d["steps"] < wall_ms
    assert d["full_scene_ms_extrapolated"] > d["ms_per_step"]
    # the same workload description as the GPU arm's line
    sys.path.insert(0, ROOT)
    import bench
    from paper_2508_03065_gb300 import workloads as W

    assert d["config"] == json.loads(json.dumps(bench.workload_config(W.config2())))


def test_parity_summary_of_the_timed_output():
    sys.path.insert(0, ROOT)
    import bench

    ref = np.linspace(-1.0, 1.0, 9)
    y = np.zeros(100)
    idx = np.arange(0, 90, 10)
    y[idx] = ref * (1 + 1e-7)
    p = bench.parity_of(y, idx, ref)
    assert p["ok"] and p["samples"] == 9 and abs(p["rel_l2"] - 1e-7) < 1e-9
    y[idx[3]] += 0.1
    assert not bench.parity_of(y, idx, ref)["ok"]
