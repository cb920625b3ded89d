"""bench.py's reference arm (the FP64 oracle on the host cores) keeps the bench line's
contract: one JSON line from rank 0 with the arm's metric, unit and direction, the
oracle described as a CPU baseline, no host-device bytes and no GPU launches; other
ranks print nothing and exit 0. CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(env_extra):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600, check=True)
    return [ln for ln in out.stdout.splitlines() if ln.strip()]


def test_reference_line():
    lines = run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "points/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "key-points" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["gpu_launches"] == 0 and d["config"]["W"] == 1242 and d["config"]["H"] == 375


def test_reference_other_ranks_are_silent():
    assert run({"RANK": "1", "WORLD_SIZE": "2"}) == []
