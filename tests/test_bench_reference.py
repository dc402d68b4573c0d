"""bench.py's reference arm on CPU: the oracle timed on a bounded sample of
the benchmark workload prints one JSON line with the fields of the other
arm (same metric, unit, direction and config), a cpu_baseline describing
the run and an e2e object with no host transfers; a rank other than 0 of a
multi-rank launch prints nothing and exits 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, args=()):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "2", "--warmup", "1", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_contract_line():
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == "sparse-gate terms/s" and line["unit"] == "terms/s"
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["value"] > 0
    cfg = line["config"]
    assert (cfg["n"], cfg["K"], cfg["p"], cfg["seed"]) == (60, 1 << 26, 0.9999, 1003)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert "gates 1.." in cb["sample"]
    e2e = line["e2e"]
    assert e2e == {"value": line["value"], "unit": "terms/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, ("--gpus", "2"))
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
