"""The oracle and the CUDA path share no code (CPU, static): the package never imports the
oracle, the oracle takes only the seeded input generators (workloads.py) from the package,
neither side includes the other's C or CUDA sources, the input generators import neither
side, bench.py reaches the oracle only from its CPU-baseline and reference legs, and the
entry-point module only to build it and in smoke()."""
import ast
import glob
import os
import re

from tests.conftest import ROOT

PKG = os.path.join(ROOT, "paper_2107_01745_b300")
ORACLE = os.path.join(ROOT, "oracle")


def _imports(path):
    """(module name, enclosing top-level function or None) of every import in a Python file,
    plus string arguments of importlib.import_module / __import__ calls."""
    tree = ast.parse(open(path).read(), filename=path)
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) and fn is None else fn
            if isinstance(child, ast.Import):
                out.extend((a.name, f) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                base = "." * child.level + (child.module or "")
                out.append((base, f))
                out.extend((f"{base}.{a.name}", f) for a in child.names)
            elif isinstance(child, ast.Call) and getattr(child.func, "attr", getattr(child.func, "id", "")) in (
                    "import_module", "__import__"):
                out.extend((a.value, f) for a in child.args if isinstance(a, ast.Constant) and isinstance(a.value, str))
            visit(child, f)

    visit(tree, None)
    return out


def _py(root):
    return [p for p in glob.glob(os.path.join(root, "**", "*.py"), recursive=True) if "_build" not in p]


def test_package_never_imports_the_oracle():
    for path in _py(PKG):
        for name, _ in _imports(path):
            assert not re.match(r"(\.+)?oracle\b", name), f"{os.path.relpath(path, ROOT)} imports {name}"


def test_oracle_takes_only_the_input_generators_from_the_package():
    for path in _py(ORACLE):
        for name, _ in _imports(path):
            if name.startswith("paper_2107_01745_b300"):
                assert name.startswith("paper_2107_01745_b300.workloads") or name == "paper_2107_01745_b300", \
                    f"{os.path.relpath(path, ROOT)} imports {name}"


def test_input_generators_import_neither_side():
    for name, _ in _imports(os.path.join(PKG, "workloads.py")):
        assert not re.match(r"(oracle|paper_2107_01745_b300\.(stotree|warmstart|build)|ctypes|torch)\b", name), name


def test_no_shared_c_or_cuda_sources():
    cuda = glob.glob(os.path.join(PKG, "csrc", "*"))
    c_oracle = glob.glob(os.path.join(ORACLE, "*.c")) + glob.glob(os.path.join(ORACLE, "*.h"))
    assert cuda and c_oracle
    for path in cuda:
        for inc in re.findall(r'#\s*include\s*[<"]([^">]+)[">]', open(path, errors="replace").read()):
            assert "oracle" not in inc, f"{path} includes {inc}"
    for path in c_oracle:
        for inc in re.findall(r'#\s*include\s*[<"]([^">]+)[">]', open(path).read()):
            assert inc in {"math.h", "stdlib.h", "string.h", "omp.h", "stdint.h", "stddef.h"}, f"{path} includes {inc}"


def test_bench_reaches_the_oracle_only_from_its_cpu_legs():
    users = {fn for name, fn in _imports(os.path.join(ROOT, "bench.py")) if name.split(".")[0] == "oracle"}
    assert users and users <= {"cpu_baseline", "run_reference"}, users


def test_entry_points_reach_the_oracle_only_to_build_it_and_in_smoke():
    """build() compiles the C oracle beside the library (building the checker, not using it);
    smoke() checks one small run against it."""
    users = {fn for name, fn in _imports(os.path.join(ROOT, "__graft_entry__.py")) if name.split(".")[0] == "oracle"}
    assert users <= {"build", "smoke"}, users
