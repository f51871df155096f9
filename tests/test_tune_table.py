"""The autotuner's launch-shape table (host side, no GPU): JSON save / load round
trip, replacement of entries with the same key, lookups by size class, and rejection
of malformed or out-of-range files without touching the table."""
import json
import os

import pytest


@pytest.fixture()
def bem():
    b = pytest.importorskip("paper_2206_00708_gb300")
    b.bem_tune_clear()
    yield b
    b.bem_tune_clear()


def _write(path, entries, fmt="bem-tune-1"):
    with open(path, "w") as fh:
        json.dump({"format": fmt, "entries": entries}, fh)


def test_load_lookup_save_round_trip(bem, tmp_path):
    src = tmp_path / "a.json"
    _write(src, [{"kernel": "cheb", "width": 1, "n_log2": 16, "block": 256, "variant": 0, "ms": 1.07},
                 {"kernel": "cheb", "width": 8, "n_log2": 16, "block": 128, "variant": 0, "ms": 0.02},
                 {"kernel": "gemm_tc", "width": 64, "n_log2": 14, "block": 0, "variant": 1, "ms": 0.6}])
    bem.bem_tune_load(str(src))
    assert bem.bem_tune_count() == 3
    # rows in (2^15, 2^16] share the size class 16
    assert bem.bem_tune_get("cheb", 1, 40968)[:2] == (256, 0)
    assert bem.bem_tune_get("cheb", 1, 65536)[:2] == (256, 0)
    assert bem.bem_tune_get("cheb", 1, 65537)[0] == 0  # no entry: the kernel's default
    assert bem.bem_tune_get("cheb", 8, 40968)[:2] == (128, 0)
    assert bem.bem_tune_get("cheb", 8, 200000)[0] == 0
    assert bem.bem_tune_get("gemm_tc", 64, 10248)[:2] == (0, 1)
    out = tmp_path / "b.json"
    bem.bem_tune_save(str(out))
    data = json.loads(out.read_text())
    assert data["format"] == "bem-tune-1" and len(data["entries"]) == 3
    bem.bem_tune_clear()
    assert bem.bem_tune_count() == 0
    bem.bem_tune_load(str(out))
    assert bem.bem_tune_get("cheb", 8, 50000)[:2] == (128, 0)
    b, v, ms = bem.bem_tune_get("cheb", 1, 40968)
    assert (b, v) == (256, 0) and abs(ms - 1.07) < 1e-9


def test_load_replaces_entries_with_the_same_key(bem, tmp_path):
    p = tmp_path / "c.json"
    _write(p, [{"kernel": "cheb", "width": 8, "n_log2": 12, "block": 128, "variant": 0}])
    bem.bem_tune_load(str(p))
    _write(p, [{"kernel": "cheb", "width": 8, "n_log2": 12, "block": 64, "variant": 0}])
    bem.bem_tune_load(str(p))
    assert bem.bem_tune_count() == 1
    assert bem.bem_tune_get("cheb", 8, 4000)[:2] == (64, 0)


@pytest.mark.parametrize("entries,fmt", [
    ([{"kernel": "cheb", "width": 1, "n_log2": 16, "block": 96, "variant": 0}], "bem-tune-1"),
    ([{"kernel": "cheb", "width": 1, "n_log2": 16, "block": 256, "variant": 3}], "bem-tune-1"),
    ([{"kernel": "nope", "width": 1, "n_log2": 16, "block": 256, "variant": 2}], "bem-tune-1"),
    ([{"kernel": "cheb", "width": 1, "n_log2": 16, "variant": 0}], "bem-tune-1"),
    ([{"kernel": "cheb", "width": 1, "n_log2": 16, "block": 64, "variant": 0}], "other"),
    ([{"kernel": "cheb", "width": "one", "n_log2": 16, "block": 64, "variant": 0}], "bem-tune-1"),
    ([{"kernel": "cheb", "width": 1, "n_log2": 16, "block": 99999999999999999999, "variant": 0}], "bem-tune-1"),
])
def test_malformed_files_are_rejected_and_merge_nothing(bem, tmp_path, entries, fmt):
    p = tmp_path / "bad.json"
    _write(p, entries, fmt)
    with pytest.raises(bem.BemError) as e:
        bem.bem_tune_load(str(p))
    assert e.value.status == bem.BEM_E_INVALID_ARG
    assert bem.bem_tune_count() == 0
    with pytest.raises(bem.BemError):
        bem.bem_tune_load(str(tmp_path / "missing.json"))


def test_tuning_file_named_in_the_environment_is_loaded_with_the_library(tmp_path):
    """BEM_TUNE_FILE: the table of a fresh process starts with that file's entries."""
    import os
    import subprocess
    import sys
    p = tmp_path / "env.json"
    _write(p, [{"kernel": "gemm_tc", "width": 64, "n_log2": 14, "block": 0, "variant": 2, "ms": 2.5}])
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import paper_2206_00708_gb300 as b; "
            "print(b.bem_tune_count(), b.bem_tune_get('gemm_tc', 64, 10000)[:2])")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                         env=dict(os.environ, BEM_TUNE_FILE=str(p)), timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "1 (0, 2)", out.stdout
