"""Static checks of the separation between the product and its checker (no GPU).

The CUDA path (the package) and the CPU oracle share no code: neither imports
or includes the other, and the seeded input generators (ew_inputs.py) import
neither.  Outside the tests, only smoke() and bench.py's CPU-baseline and
reference legs touch the oracle.  Without its compiled library the package
does not import: there is no fallback.
"""
import ast
import os
import re
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2507_18282_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for d, _, files in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _imports_and_includes(path):
    src = open(path, encoding="utf-8").read()
    return re.findall(r"^\s*(?:from\s+\S+\s+import|import\s+\S+|#\s*include\s*[<\"][^>\"]+[>\"]).*$", src, flags=re.M)


def test_package_never_reaches_the_oracle():
    for f in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        for line in _imports_and_includes(f):
            assert "oracle" not in line, (f, line)


def test_oracle_never_reaches_the_package():
    for f in _sources(ORACLE, (".py", ".c", ".h")):
        for line in _imports_and_includes(f):
            assert not re.search(r"paper_2507_18282_gb300|csrc|ew_internal|ew_[a-z0-9_]*\.cuh|\bew\.h\b", line), (f, line)


def test_input_generators_import_neither_side():
    for line in _imports_and_includes(os.path.join(ROOT, "ew_inputs.py")):
        assert "oracle" not in line and "paper_2507_18282_gb300" not in line, line


def _oracle_import_sites(path):
    """(enclosing function, enclosing if-tests) of every import of the oracle."""
    tree = ast.parse(open(path, encoding="utf-8").read())
    sites = []

    def walk(node, fn, tests):
        for child in ast.iter_child_nodes(node):
            if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)):
                walk(child, child.name, [])
            elif isinstance(child, ast.If):
                walk(child, fn, tests + [ast.unparse(child.test)])
            else:
                if isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                    sites.append((fn, tests))
                if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                    sites.append((fn, tests))
                walk(child, fn, tests)
    walk(tree, None, [])
    return sites


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    sites = _oracle_import_sites(os.path.join(ROOT, "bench.py"))
    assert sites
    for fn, tests in sites:
        # _oracle_sample_worker: one process of the all-cores CPU baseline
        assert fn in ("cpu_baseline_sample", "_oracle_sample_worker", "run_reference", "run_ours"), fn
        if fn == "run_ours":
            assert any("no_cpu_baseline" in t for t in tests), tests


def test_graft_entry_uses_the_oracle_only_to_build_it_and_in_smoke():
    for fn, _ in _oracle_import_sites(os.path.join(ROOT, "__graft_entry__.py")):
        assert fn in ("build", "smoke"), fn


def test_package_without_its_library_does_not_import(tmp_path):
    dst = tmp_path / "paper_2507_18282_gb300"
    dst.mkdir()
    for f in os.listdir(PKG):
        if f.endswith(".py"):
            shutil.copy(os.path.join(PKG, f), dst / f)
    r = subprocess.run([sys.executable, "-c", "import paper_2507_18282_gb300"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "not built" in r.stderr
