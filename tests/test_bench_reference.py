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


def test_every_traced_kernel_has_a_work_model():
    """Each name the library traces (Trace(stream, "name") in csrc) has an
    algorithmic work model in bench.kernel_work, or a stated reason in
    bench.NO_MODEL, so that every kernel of the step gets a roofline entry."""
    import re
    sys.path.insert(0, ROOT)
    import bench
    csrc = os.path.join(ROOT, "paper_2505_06932_gb300", "csrc")
    names = set()
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh")):
            names |= set(re.findall(r'Trace\s+\w+\(\s*[\w>.\-]+\s*,\s*"([^"]+)"\s*\)', open(os.path.join(csrc, f)).read()))
    assert {"k_ppic_acc<float>", "k_clip32", "k_csf_force", "k_csf_ring_list"} <= names
    w = dict(T=1000, V=500, N=64 ** 3, C=5000, P=4000, M=300, ring=350, fit_pairs=120000, clip_f64=20)
    missing = []
    for n in sorted(names):
        models = [bench.kernel_work(n, w, fp32) for fp32 in (False, True)]
        if n in bench.NO_MODEL:
            continue
        if any(m is None for m in models):
            missing.append(n)
            continue
        for bound, work, text in models:
            assert bound in ("hbm", "fp32", "fp64") and work > 0 and text, n
    assert not missing, missing
