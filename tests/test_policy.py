"""Separation of the product path from the oracle (CPU only): nothing in the library
package or the shared input generators imports the oracle, the CUDA sources do not
reference it, and bench.py imports it only inside its CPU-baseline sample (the
pool task that the `cpu_baseline` and `--impl reference` legs run)."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read())
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [(a.name, node) for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append((node.module, node))
    return tree, out


def test_library_and_inputs_never_import_the_oracle():
    for d in ("paper_2206_00708_gb300", "bem_inputs"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, d)):
            for f in files:
                if f.endswith(".py"):
                    _, imps = _imports(os.path.join(dirpath, f))
                    assert not any(m == "oracle" or m.startswith("oracle.") for m, _ in imps), (dirpath, f)
                if f.endswith((".cu", ".cuh", ".h", ".c")):
                    assert "oracle" not in open(os.path.join(dirpath, f)).read(), (dirpath, f)


def test_bench_imports_the_oracle_only_in_its_cpu_sample():
    tree, imps = _imports(os.path.join(ROOT, "bench.py"))
    parents = {}
    for node in ast.walk(tree):
        for child in ast.iter_child_nodes(node):
            parents[child] = node
    for mod, node in imps:
        if mod == "oracle" or mod.startswith("oracle."):
            p = parents.get(node)
            while p is not None and not isinstance(p, ast.FunctionDef):
                p = parents.get(p)
            assert p is not None and p.name == "_oracle_task", (mod, getattr(p, "name", None))
