"""The benchmark's reference arm (the CPU FP64 oracle on bounded samples of
the default workload) keeps the JSON contract of the GPU arm: one line with
the same metric, unit, direction and workload, its CPU baseline described,
and an end-to-end entry without host-device copies; under a multi-rank
launcher only rank 0 runs it.  No GPU."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.strip()]


def _bench_constants():
    spec = importlib.util.spec_from_file_location("bench_consts", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv, sys.argv = sys.argv, ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_reference_arm_prints_one_contract_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    b = _bench_constants()
    assert d["impl"] == "reference"
    assert (d["metric"], d["unit"], d["higher_is_better"]) == ("solves/s", "solves/s", True)
    assert d["config"]["workload"] == b.WORKLOAD_DESC
    assert d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    assert abs(d["ms_per_step"] - 1000.0 / d["value"]) <= 1e-9 * d["ms_per_step"]
    # every timed step solved a whole window: the steps fit in the timed wall time
    wall = float(d["cpu_baseline"]["sample"].rsplit("timed wall ", 1)[1].split()[0])
    assert d["steps"] * d["ms_per_step"] <= 1e3 * wall + 100.0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_on_other_ranks():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
