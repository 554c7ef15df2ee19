"""The product path and the oracle stay apart, and the product path has no
fallback: a static scan of the package for any use of the oracle, and the
binding refusing to run without its native library."""

import ast
import os

import pytest

from paper_1102_3069_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1102_3069_gb300")


def _package_files(exts):
    for d, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_python_never_imports_the_oracle():
    for path in _package_files((".py",)):
        tree = ast.parse(open(path).read(), path)
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            else:
                continue
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (path, names)


def test_native_sources_never_reach_the_oracle():
    for path in _package_files((".cu", ".cuh", ".h", ".cpp", ".c")):
        text = open(path).read()
        assert "oracle/" not in text and "#include \"oracle" not in text, path


def test_binding_refuses_to_run_without_its_library(monkeypatch):
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", os.path.join(PKG, "no_such_libmm.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        B.lib()
