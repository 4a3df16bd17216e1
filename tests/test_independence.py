"""The FP64 oracle and the CUDA path stay apart.

The parity tests mean something only if the two sides share no code. The product package never
imports the oracle. The oracle imports nothing of the package and stays plain numpy. The CUDA
sources include nothing from it. Outside `tests/`, the oracle is imported only by the smoke check
and by the benchmark's CPU-baseline sample, which the reference arm also times.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1905_12725_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _py_files(folder):
    for dirpath, _, names in os.walk(folder):
        if "__pycache__" in dirpath or "_build" in dirpath:
            continue
        for n in names:
            if n.endswith(".py"):
                yield os.path.join(dirpath, n)


def _imports(path):
    """(module name, enclosing top-level function or None) for every import in a file."""
    tree = ast.parse(open(path, encoding="utf-8").read(), filename=path)
    out = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = func
            if func is None and isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)):
                f = child.name
            if isinstance(child, ast.Import):
                out.extend((a.name, f) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                if child.level == 0 and child.module:
                    out.append((child.module, f))
                elif child.level > 0:
                    out.append(("." * child.level + (child.module or ""), f))
            visit(child, f)

    visit(tree, None)
    return out


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        for mod, _ in _imports(path):
            assert mod.split(".")[0] != "oracle", f"{path} imports {mod}"


def test_oracle_is_plain_numpy_and_imports_nothing_of_the_package():
    allowed = {"__future__", "math", "numpy", "oracle", "."}
    files = list(_py_files(ORACLE))
    assert files
    for path in files:
        for mod, _ in _imports(path):
            root = mod.split(".")[0] if not mod.startswith(".") else "."
            assert root in allowed, f"{path} imports {mod}"


def test_cuda_sources_include_nothing_from_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', re.M)
    names = [n for n in os.listdir(csrc) if n.endswith((".cu", ".cuh", ".h"))]
    assert names
    for n in names + [os.path.join(os.pardir, os.pardir, "include", "dbfft.h")]:
        text = open(os.path.join(csrc, n), encoding="utf-8").read()
        for target in inc.findall(text):
            assert "oracle" not in target, f"{n} includes {target}"


def test_oracle_is_imported_only_by_the_smoke_check_and_the_cpu_baseline():
    expected = {
        os.path.join(ROOT, "__graft_entry__.py"): {"smoke"},
        os.path.join(ROOT, "bench.py"): {"oracle_sample", "_oracle_rhs_job"},  # the CPU baseline (1 core, all cores)
    }
    for path, funcs in expected.items():
        users = {f for mod, f in _imports(path) if mod.split(".")[0] == "oracle"}
        assert users == funcs, f"{path}: oracle imported in {users or 'no function'}"
