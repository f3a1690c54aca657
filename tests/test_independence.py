"""The library and the oracle stay independent (CPU only, reads source text).

* Nothing in the package, the C headers or the CUDA sources imports, loads or names the
  oracle: the product path has no CPU fallback through it.
* The oracle imports nothing of the package but the seeded input generators
  (``workloads``, which hold none of the method's arithmetic), and nothing compiled.
* The package's Python code imports no test module, and nothing committed reads scratch
  files outside the repository's tracked tree.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1406_7803_gb300")


def _files(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if not x.startswith((".", "_", "build")) and x != "__pycache__"]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            mod = ("." * node.level) + (node.module or "")
            yield mod
            for a in node.names:
                yield mod + "." + a.name


def test_package_never_touches_the_oracle():
    for f in _files(PKG, (".py",)):
        for name in _imports(f):
            assert name.split(".")[0] not in ("oracle", "tests"), (f, name)
        tree = ast.parse(open(f).read(), f)
        for node in ast.walk(tree):
            if isinstance(node, ast.Name):
                assert node.id != "oracle", (f, node.lineno)
            if isinstance(node, ast.Constant) and isinstance(node.value, str):
                assert "oracle/" not in node.value and node.value != "oracle", (f, node.lineno)
    for f in list(_files(PKG, (".cu", ".cuh", ".h", ".cpp"))) + list(_files(os.path.join(ROOT, "include"), (".h",))):
        for line in open(f):
            if line.lstrip().startswith("#include"):
                assert "oracle" not in line, (f, line)
            assert "oracle/" not in line, (f, line)


def test_oracle_imports_only_the_input_generators():
    for f in _files(os.path.join(ROOT, "oracle"), (".py",)):
        for name in _imports(f):
            top = name.split(".")[0]
            if top == "paper_1406_7803_gb300":
                assert name in ("paper_1406_7803_gb300", "paper_1406_7803_gb300.workloads"), (f, name)
            assert top not in ("ctypes", "torch", "tests"), (f, name)
        text = open(f).read()
        assert "libfde" not in text and "fde.py" not in text, f


def test_no_committed_code_reads_scratch_files():
    paths = list(_files(PKG, (".py", ".cu", ".cuh", ".h"))) + list(_files(os.path.join(ROOT, "oracle"), (".py",)))
    paths += list(_files(os.path.join(ROOT, "tests"), (".py",)))
    paths += [os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")]
    for f in paths:
        if os.path.abspath(f) == os.path.abspath(__file__):
            continue
        text = open(f).read()
        assert "_work/" not in text, f
