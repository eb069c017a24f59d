"""bench.py --impl reference: the oracle timed on the host cores, one JSON line with the GPU arm's
metric and unit, a cpu_baseline describing the run and an e2e object with no copies; under a
multi-rank launch only rank 0 runs and prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, **env):
    e = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    e.update(env)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], env=e, capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    return r


def test_reference_arm_line():
    r = run(["--impl", "reference", "--config", "deconv1d", "--steps", "2", "--warmup", "1",
             "--cpu-sample-iters", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "iterations/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1
    assert "deconv1d" in line["metric"] and line["config"]["workload"].startswith("deconv1d")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and "3 iterations" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_are_silent():
    r = run(["--impl", "reference", "--config", "deconv1d", "--steps", "1", "--warmup", "1",
             "--cpu-sample-iters", "3"], RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_reference_arm_batch_line():
    """The CT batch's oracle arm: one single-threaded process per host core, each on its own
    instance, instance-iterations/s with the GPU arm's metric (a 48 x 48 image keeps it short)."""
    r = run(["--impl", "reference", "--ct-size", "48", "--steps", "1", "--warmup", "1",
             "--cpu-sample-iters", "12"])
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "instance-iterations/s" and line["value"] > 0
    assert line["config"]["workload"].startswith("ct2d_batch: 48x48")
    cb = line["cpu_baseline"]
    assert cb["cores"] == (os.cpu_count() or 1) and cb["value"] == line["value"] and "3 iterations" in cb["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
