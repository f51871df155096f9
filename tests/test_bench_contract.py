"""The bench's last output line: built from stub measurements, it parses as JSON, is
the last line printed, stays under the size limit and carries every contract key."""
import io
import json
import os
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stub_line():
    roof = {"kernel": "k_tile<float2,1>", "bound": "hbm", "achieved": 6012.345678, "peak": 6791.7, "unit": "GB/s",
            "frac": 0.88527, "traffic": 3.3712345e9, "peak_kind": "measured", "algorithmic_bytes_per_launch": 3.36e9,
            "avg_launch_ms": 0.5591234}
    roof2 = {"kernel": "k_regular32<false>", "bound": "alu", "achieved": 15.2345, "peak": 80.54, "unit": "TFLOP/s",
             "frac": 0.18912, "traffic": None, "flop_per_point_pair": 91, "point_pairs_per_launch": 7.5e9,
             "avg_launch_ms": 52.0123}
    fp64 = {"value": 0.2634567, "times": [3801.2, 3799.9, 3802.5]}
    err = {"v_ext": 2.4e-7, "w_ext": 9.6e-7, "v_int": 3.1e-7, "w_int": 5.5e-7}
    cpu = {"value": 3.7e-4, "cores": 16, "sample_short": "extrapolated from ~190 test triangles + a 512-row "
                                                        "matvec block x 205 iterations"}
    e2e = {"value": 1.8312345, "h2d_bytes_per_step": 737424, "d2h_bytes_per_step": 655488}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 55}
    return bench.contract_line(value=1.8123456, steps=20, warmup=5, world=1, times=[551.2] * 19 + [560.9],
                               clocks=clocks, launches=7745 * 20, err=err, fp64=fp64, roof=roof, roof2=roof2,
                               cpu=cpu, e2e=e2e)


def test_contract_line_is_last_compact_and_complete():
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.emit_section("serving", {"workload": "x" * 5000, "saturated": {"mixed": {"solves_per_s": 8.0}}})
        bench.emit_section("kernels", [{"name": "k", "ms": 1.0, "launches": 3}])
        bench.emit_contract(_stub_line())
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 3
    for ln in lines:
        json.loads(ln)
    last = lines[-1]
    assert len(last.encode()) <= bench.CONTRACT_MAX_BYTES, len(last)
    d = json.loads(last)
    assert "section" not in d
    for key in bench.CONTRACT_KEYS:
        assert key in d, key
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in d["roofline"], key
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in d["cpu_baseline"], key
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in d["e2e"], key
    for key in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert key in d["clocks"], key
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["value"] > 0
    assert d["latency_ms"]["p50"] <= d["latency_ms"]["p99"]
    assert d["config"]["workload"]


def test_flop_count_is_the_stated_table():
    assert bench.FLOP_PER_POINT_PAIR == sum(f for _, f in bench.FLOP_COUNT_PER_POINT_PAIR)
    assert 80 <= bench.FLOP_PER_POINT_PAIR <= 120
