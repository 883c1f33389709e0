"""The benchmark's reference arm (the oracle on the host cores) keeps the
one-line JSON contract: it runs without a GPU, prints one line with the
metric, the unit, the cpu_baseline and e2e objects, marks itself
"impl": "reference", prints an "unavailable" line for the workload that has
no CPU counterpart, and leaves every rank but 0 silent."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=e,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.strip()]


@pytest.mark.parametrize("workload,unit", [("one256", "Mpixel/s"), ("exhaustive", "fits/s")])
def test_reference_line(workload, unit):
    lines = run_bench("--workload", workload, "--steps", "2", "--warmup", "1", "--ref-step-s", "0.5")
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == unit and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith(workload)


def test_serving_has_no_cpu_counterpart():
    lines = run_bench("--workload", "serving", "--steps", "1", "--warmup", "0")
    d = json.loads(lines[-1])
    assert d["impl"] == "reference" and "unavailable" in d


def test_other_ranks_print_nothing():
    assert run_bench("--steps", "1", "--warmup", "0", env={"RANK": "1", "WORLD_SIZE": "2"}) == []
