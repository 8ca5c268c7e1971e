"""The oracle and the CUDA path share no code: the oracle's C source includes
only the C library, no CUDA source or the C header names the oracle, the
package never imports the oracle module, and bench.py loads it only inside its
CPU-baseline function."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1909_06374_gb300")


def test_oracle_c_includes_only_the_c_library():
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    includes = re.findall(r'#\s*include\s*([<"][^>"]+[>"])', src)
    assert includes, "no includes found"
    for inc in includes:
        assert inc.startswith("<"), inc           # no project header
        assert "agnlc" not in inc and "lc_" not in inc, inc


def test_cuda_sources_never_name_the_oracle():
    for path in glob.glob(os.path.join(PKG, "csrc", "*")) + [os.path.join(ROOT, "include", "agnlc.h")]:
        src = open(path).read()
        assert "oracle" not in src.lower(), path
        for inc in re.findall(r'#\s*include\s*"([^"]+)"', src):
            assert "oracle" not in inc, (path, inc)


def _top_level_imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in tree.body:
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            names.add(node.module.split(".")[0])
    return names


def _all_imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            names.add(node.module.split(".")[0])
    return names


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        assert "oracle" not in _all_imports(path), path


def test_bench_loads_the_oracle_only_for_its_cpu_baseline():
    path = os.path.join(ROOT, "bench.py")
    assert "oracle" not in _top_level_imports(path)
    tree = ast.parse(open(path).read())
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
                    users.add(fn.name)
    assert users == {"cpu_baseline_run"}, users
