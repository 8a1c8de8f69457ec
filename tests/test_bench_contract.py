"""bench.py's reference arm (the oracle timed on host cores) runs without a GPU and
prints one JSON line with the contract's keys; too few warm-up steps are refused."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, timeout=600, cwd=ROOT)


def _line(*args):
    r = _bench("--impl", "reference", *args)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_default_is_the_large_network_sampled():
    """The default workload is the 200,000-stop network with 1,024 queries per step; the
    oracle runs a bounded sample of each step's batch, and the line says so."""
    d = _line("--steps", "1", "--warmup", "3")
    assert d["config"]["global_batch"] == 1024 and d["config"]["n_stops"] == 200000
    assert "first 64 queries of each 1,024-query step" in d["cpu_baseline"]["sample"]
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]


def test_reference_arm_line():
    r = _bench("--impl", "reference", "--workload", "city", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["global_batch"] == 256 and d["config"]["n_stops"] == 20000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_too_few_warmup_steps_refused():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "2")
    assert r.returncode != 0
