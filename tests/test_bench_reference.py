"""bench.py's oracle arm (--impl reference) on CPU: it keeps the launch contract (K timed
steps after W >= 3 untimed ones, one JSON line with the GPU arm's metric, unit and
config) and describes its own run in cpu_baseline and e2e."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3", "--warmup", "1",
           "--images", "12", "--size", "48", "--reference-budget", "2"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "Mpixel/s encode+decode (bit-exact)" and d["unit"] == "Mpixel/s"
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["steps"] == 3 and d["warmup"] == 3                     # W is raised to 3
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["H"] == 48 and d["config"]["images_per_gpu"] == 12
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "per step" in cb["sample"] and "3 timed steps" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # throughput and step time describe the same steps: a whole number of images per
    # step, at least one per core
    m = d["value"] * 1e6 * d["ms_per_step"] / 1e3 / (48 * 48)
    assert abs(m - round(m)) < 1e-6 and round(m) >= cb["cores"]
    assert cb["sample"].startswith(f"{round(m)} of the workload's 48x48 images per step")


def test_reference_arm_other_ranks_do_nothing():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--images", "4",
           "--size", "32"]
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""
