"""The ctypes structures of the Python binding have the layout of the C structures
of include/bem.h: a small C program built with the host compiler prints sizeof and
every field's offsetof, and each must equal the ctypes value (CPU only)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _structs(bem):
    return {name: getattr(bem, name) for name in ("bem_c128", "bem_incident", "bem_solve_opts", "bem_solve_report",
                                                  "bem_instance", "bem_server_opts", "bem_request", "bem_result",
                                                  "bem_serve_stats")}


def test_struct_layouts_match_the_header(tmp_path):
    bem = pytest.importorskip("paper_2206_00708_gb300")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = _structs(bem)
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bem.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            name, field, val = line.split()
            got[(name, field)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
