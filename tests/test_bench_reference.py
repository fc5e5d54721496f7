"""The benchmark's CPU legs (no GPU): the reference arm prints one JSON line of
the contract with the oracle's five steps timed, and the CPU baseline times
whole passes of the oracle over the workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "cpu_baseline", "e2e", "config"):
        assert k in line, k
    assert line["value"] > 0 and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_cpu_baseline_whole_passes():
    sys.path.insert(0, ROOT)
    import bench
    fronts = bench.workload()
    cells, times = bench.oracle_pass(fronts[1])
    assert cells > 10000 and set(times) == set(bench.PHASES)
    cb = bench.cpu_baseline(fronts, budget_s=0.0, one_core_budget_s=0.0)  # one pass over both fronts
    assert cb["value"] > 0 and cb["kind"] == "oracle" and cb["sample"].startswith("1 pass of")
    assert "one_core" not in cb


def test_cpu_baseline_one_core():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2505_06932_gb300 import inputs as I
    cb = bench.cpu_baseline([I.laplace_droplet_32(1)], budget_s=0.0, one_core_budget_s=0.1)
    one = cb["one_core"]
    assert one["cores"] == 1 and one["value"] > 0 and one["kind"] == "oracle"
