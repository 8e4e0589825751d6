"""bench.py's output contract on a GPU: one JSON line with the keys and
consistency rules the measurement relies on (a short run, small batch)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_prints_one_consistent_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "20", "--warmup", "3",
           "--batch", "4", "--no-precision", "--no-mixed", "--no-merge", "--serve-seconds", "0",
           "--cpu-seconds", "0.5", "--e2e-steps", "1", "--tune-iters", "0"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 20 and d["warmup"] >= 3
    assert d["unit"] == "GB/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["gpu_launches"] == d["steps"]  # one persistent launch per step
    # value = algorithmic bytes of the timed steps / their time
    pair_bytes = 2 * 2048 * 2048 * 4
    assert d["value"] == pytest.approx(4 * pair_bytes / (d["ms_per_step"] * 1e-3) / 1e9,
                                       rel=1e-3)
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert r["algorithmic_bytes"] == 4 * pair_bytes
    if r["traffic"] is not None:  # a profiled figure, scaled to this launch
        assert r["algorithmic_bytes"] <= r["traffic"] < 1.1 * r["algorithmic_bytes"]
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0 and c["sample"]
    e = d["e2e"]
    assert e["unit"] == "GB/s" and e["value"] > 0
    assert e["h2d_bytes_per_step"] == 4 * pair_bytes
    assert e["d2h_bytes_per_step"] == 4 * 2 * 32 * 32 * 4
    assert d["config"]["N"] == 2048 and d["config"]["N_T"] == 64
    assert d["config"]["pairs_per_step"] == 4
