"""The C example of the library (paper_2206_00708_gb300/examples/solve_octahedron.c)
compiles against include/bem.h and links against the in-tree libbem.so with the host
compiler, as a C user would build it (CPU only: it is not run here)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2206_00708_gb300")


def test_c_example_compiles_and_links(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pytest.importorskip("paper_2206_00708_gb300")  # the library is built and loads
    src = os.path.join(PKG, "examples", "solve_octahedron.c")
    exe = tmp_path / "solve_octahedron"
    p = subprocess.run([cc, "-std=c11", "-O2", "-Wall", "-Werror", src, "-I", os.path.join(ROOT, "include"),
                        "-L", PKG, "-lbem", "-Wl,-rpath," + PKG, "-o", str(exe)], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
