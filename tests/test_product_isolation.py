"""The product path has one implementation, the CUDA library: it never imports the
oracle, and without the built library it raises instead of computing anything else."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2411_14631_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield node.module or ""


def test_package_never_imports_the_oracle():
    for f in sorted(os.listdir(PKG)):
        if f.endswith(".py"):
            for name in _imports(os.path.join(PKG, f)):
                assert not name.split(".")[0] == "oracle", (f, name)


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_2411_14631_gb300 import abi
    monkeypatch.setattr(abi, "_lib", None)
    monkeypatch.setattr(abi, "LIB_PATH", str(tmp_path / "libamrhydro.so"))
    with pytest.raises(RuntimeError, match="not built"):
        abi.lib()
