"""The bench's reference arm (the oracle timed on the host's cores) runs on a
CPU and prints the one JSON line the benchmark contract asks for (no GPU
needed; the 10^3 cube workload keeps it to seconds), and the oracle leg of
the CPU baseline reports a whole solve of its workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--workload", "cube10"],
                       capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["unit"] == "s" and d["steps"] == 2
    # the value is in the metric's unit: the sample's time scaled to the
    # oracle's own iteration count; ms_per_step is what one step took
    assert d["iterations"] >= 3 and d["full_solve_s"] > 0
    assert d["ms_per_step"] < 1e3 * d["value"] * 3 / d["iterations"] * 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_cpu_leg_solves_the_whole_workload():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-leg",
                        "--workload", "cube10"], capture_output=True, text=True, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert d["dofs"] == 3993 and d["rel_resid"] <= 1e-8 and d["iterations"] > 0
    assert d["solve_s"] > 0 and d["setup_s"] > 0
