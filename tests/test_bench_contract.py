"""bench.py's reference arm (the oracle on the host) prints one JSON line with
the keys the measurement contract asks for; runs on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


def test_too_few_warmup_steps_are_rejected():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "1")
    assert r.returncode != 0 and "warmup" in r.stderr


def test_zero_lanes_are_rejected():
    r = _run("--steps", "1", "--warmup", "3", "--lanes", "0")
    assert r.returncode != 0 and "lanes" in r.stderr


def test_unknown_form_is_rejected():
    r = _run("--steps", "1", "--warmup", "3", "--forms", "batch,nothing")
    assert r.returncode != 0 and "--forms" in r.stderr
