"""bench.py --impl reference (the FP64 oracle timed on the host) prints one JSON line
with the contract's keys, on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0.0 and d["unit"] == "solves/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the value is an extrapolation from a bounded sample, and says so; ms_per_step is the
    # measured time of one sampled step (it fits the run), the extrapolated solve time is
    # given separately
    assert d["extrapolated"] is True and "extrapolated" in d["cpu_baseline"]["sample"]
    assert d["ms_per_solve_extrapolated"] > d["ms_per_step"]
    assert d["cpu_baseline"]["one_core_value"] > 0.0
