"""bench.py's CPU-side contract: the reference arm (the oracle on the host cores) prints one
JSON line with the required keys, and declines workloads whose input vector the oracle cannot
hold in host memory.  No GPU is used."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--workload", "heisenberg_ring12_full", "--steps", "2", "--warmup", "3")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "heisenberg_ring12_full"


def test_reference_arm_samples_rows_of_the_large_sector():
    """The 9,075,135,300-row sector: the oracle cannot hold its input vector, so each reference
    step is an H v on randomly sampled rows whose inputs it regenerates from their Philox index."""
    d = _run("--impl", "reference", "--workload", "heisenberg_6x6_sz0", "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and d["value"] > 0 and "unavailable" not in d
    assert d["config"]["dim"] == 9075135300 and "sampled rows" in d["cpu_baseline"]["sample"]


def test_warmup_floor():
    d = _run("--impl", "reference", "--workload", "heisenberg_ring12_full", "--steps", "1", "--warmup", "0")
    assert d["warmup"] == 3
