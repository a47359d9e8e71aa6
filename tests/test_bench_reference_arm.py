"""The benchmark's reference arm (the FP64 oracle on the host cores) on a small grid: one
JSON line with the benchmark's keys (a step is systems 1-2 of the sequence, POD-augmented
then plain PCG), and no output from ranks other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--grid", "12", "--systems", "2",
        "--steps", "2", "--warmup", "1"]


def run(env_extra=None):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(env_extra or {})
    return subprocess.run(ARGS, capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)


def test_reference_arm_line():
    p = run()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "systems/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    # one step = systems 1-2 of the sequence; the steps run as independent processes
    assert abs(d["value"] - 2e3 / d["ms_per_step"]) <= 1e-9 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["sample"]
    assert cb["cores"] == min(os.cpu_count(), 2) and cb["nproc"] == os.cpu_count()
    assert "POD-augmented" in cb["sample"] and "plain PCG" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["n"] == 12 ** 3 and d["config"]["workload"].startswith("diffusion3d_moving 12^3")
    assert d["config"]["l2"].startswith("inputs fit in L2")


def test_reference_arm_other_ranks_are_silent():
    p = run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
