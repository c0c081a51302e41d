"""The oracle and the CUDA path share no code, and the product path never
reaches the oracle (static checks, on CPU)."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2505_00136_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        assert "oracle" not in _imports(path), path


def test_cuda_sources_include_nothing_from_the_oracle():
    for path in glob.glob(os.path.join(PKG, "csrc", "*.cu*")) + glob.glob(os.path.join(ROOT, "include", "*.h")):
        for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(path).read()):
            assert "oracle" not in inc, (path, inc)


def test_oracle_includes_nothing_from_the_cuda_path():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")):
        for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(path).read()):
            assert inc in ("oracle.h", "math.h", "stdlib.h", "string.h", "stdint.h", "stdio.h"), (path, inc)
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert "paper_2505_00136_gb300" not in _imports(path), path


def test_bench_reaches_the_oracle_only_in_its_cpu_baseline():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
                    users.add(fn.name)
    assert users == {"_oracle_sample"}
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert all("oracle" not in (getattr(n, "module", None) or "") and
               all(a.name != "oracle" for a in n.names) for n in top)
