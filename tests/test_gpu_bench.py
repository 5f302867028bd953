"""bench.py end to end on a small bank: every leg of the default run (timed step,
plain, FP64 and FP32-pixel mixed legs, end-to-end call, CPU baseline) and the reference arm complete and
print one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    return json.loads(lines[0])


def test_default_legs_small_bank():
    r = run_bench("--steps", "3", "--warmup", "3", "--n-templates", "20000",
                  "--plain-waves", "1", "--leg-seconds", "0.2", "--cpu-sample", "8")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "gpu_launches", "clocks", "plain", "fp64", "mixed_f32", "e2e",
                "cpu_baseline", "mixed_vs_plain", "mixed_f32_vs_plain"):
        assert key in r, key
    # the headline step replays a CUDA graph with the autotuner's launch shape
    assert r["config"]["graph"] is True
    assert r["config"]["launch"]["autotuner_trials"] >= 8
    # the comparison legs run full waves of their launches
    for leg in ("plain", "fp64"):
        assert r[leg]["launch"]["waves"] >= 1.0 or r[leg]["n_templates"] == 20000, leg
    assert r["steps"] == 3 and r["warmup"] == 3 and r["n_gpus"] == 1
    assert r["value"] > 0 and r["gpu_launches"] > 0
    assert r["roofline"]["bound"] == "alu" and 0 < r["roofline"]["frac"] < 1.5
    assert r["e2e"]["h2d_bytes_per_step"] == 20000 * 8 * 8
    assert r["cpu_baseline"]["kind"] == "oracle" and r["cpu_baseline"]["value"] > 0


def test_reference_arm_small_sample():
    r = run_bench("--impl", "reference", "--steps", "3", "--warmup", "3", "--ref-sample", "4")
    assert r["impl"] == "reference" and r["value"] > 0
    assert r["e2e"]["h2d_bytes_per_step"] == 0 and r["cpu_baseline"]["kind"] == "oracle"
