"""bench.py's reference arm (the FP64 CPU oracle timed on the host) runs without a GPU and prints
one JSON line with the keys the benchmark contract names."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def _check_contract(d):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["sample"] and cb["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_scan_reference_arm():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-seconds", "1")
    _check_contract(d)
    assert d["unit"] == "solves/s" and d["higher_is_better"] is True


def test_table_1_reference_arm_reproduces_the_papers_structure():
    """Sec. IV Table 1 on the host: four algorithms, one solution, one iteration count, and the
    modified interpolation and the parallel loop each faster than the traditional serial code."""
    d = _run("--impl", "reference", "--workload", "table1")
    _check_contract(d)
    algs = d["algorithms"]
    assert len(algs) == 4
    its = {a["iterations"] for a in algs.values()}
    a0 = {round(a["A0"], 12) for a in algs.values()}
    assert len(its) == 1 and len(a0) == 1
    t = {k.split()[0]: a["wall_s"] for k, a in algs.items()}
    assert t["2"] < t["1"] and t["4"] < t["2"]
    if d["cores"] > 1:
        assert t["3"] < t["1"]


def test_sweep_rate_and_temperature_reference_arms():
    """The oracle arms of the fixed-sweep rate (BC-kernel evaluations per second) and of the
    finite-temperature scan keep the same contract, with the units of their GPU arms."""
    d = _run("--impl", "reference", "--workload", "sweep-rate", "--cpu-seconds", "1")
    _check_contract(d)
    assert d["unit"] == "evals/s" and len(d["cpu_baseline"]["seconds_per_sweep"]) == 12
    d = _run("--impl", "reference", "--workload", "temperature", "--cpu-seconds", "1")
    _check_contract(d)
    assert d["unit"] == "solves/s" and d["cpu_baseline"]["extrapolation"] is True
