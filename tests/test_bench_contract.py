"""bench.py keeps its one-JSON-line contract: the reference arm (the FP64 oracle on the host
cores) on the CPU, and the GPU arm with every key the line must carry."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def last_json_line(out):
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = last_json_line(r.stdout)
    assert d["impl"] == "reference" and d["metric"] == "EGT iter/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_gpu_arm_line_has_every_key():
    r = subprocess.run([sys.executable, "bench.py", "--steps", "3", "--warmup", "3", "--cpu-seconds", "1",
                        "--batch-games", "4", "--batch-iters", "20", "--served-requests", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    d = last_json_line(r.stdout)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in d, k
    assert d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0 and d["gpu_launches"] == 3
    assert "workload" in d["config"]
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and 0 < rf["frac"] < 1.5
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] > 0
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert d["batched"]["value"] > 0 and d["batched"]["tuned"]["shape"]["share"] in range(5)
    assert 0 < d["batched"]["roofline"]["frac"] < 1.5
    assert d["large"]["value"] > 0 and 0 < d["large"]["roofline"]["frac"] < 1.5
    assert d["large"]["time_to_gap"]["iters"] > 0
    cf = d["cpu_fast"]
    assert cf["value"] > 0 and cf["cores"] >= 1 and cf["time_to_gap"]["iters"] > 0
    sv = d["served"]
    assert sv["requests"] == 3 and sv["solves_per_s"] > 0 and sv["latency_p99_s"] >= sv["latency_p50_s"] > 0
    assert sorted(x["rate"] for x in sv["sweep"]) == [10.0, 100.0, 500.0]
    assert all(x["requests"] == 3 and x["solves_per_s"] > 0 for x in sv["sweep"])
