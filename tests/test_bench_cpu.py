"""bench.py's host-side contract, on the CPU: the reference arm (the FP64
oracle timed on the host cores) prints one JSON line with the contract's keys;
under a multi-rank launch only rank 0 prints; fewer than 3 warm-up steps are
refused."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*argv, env_extra=None):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_json_line():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "3", "--cpu-seconds", "2")
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in j, k
    assert j["value"] > 0 and j["unit"] == "GFLOP/s" and j["higher_is_better"] is True
    assert (j["n_gpus"], j["steps"], j["warmup"]) == (1, 1, 3)
    assert j["dtype"] == "f64" and j["data"] == "synthetic" and "workload" in j["config"]
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"] and cb["sample"]
    e = j["e2e"]
    assert (e["value"], e["unit"], e["h2d_bytes_per_step"], e["d2h_bytes_per_step"]) == (j["value"], j["unit"], 0, 0)


def test_reference_arm_other_ranks_print_nothing():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "3", "--cpu-seconds", "2",
               env_extra={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_warmup_below_three_is_refused():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "2", "--cpu-seconds", "1")
    assert r.returncode != 0 and "--warmup" in r.stderr
