"""The oracle and the CUDA path share no code (no GPU needed).

* Nothing in the product package (its Python modules, CUDA sources and
  build script) imports, includes, links or loads anything under oracle/.
* The oracle imports nothing from the product package: its inputs come
  from the caller (the tests pass the seeded generators' fields).
* The C oracle includes only the C standard library.
* The product fails loudly when its CUDA library is missing: the binding
  raises, there is no CPU fallback.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2303_10499_gb300")
ORC = os.path.join(ROOT, "oracle")


def files(top, exts):
    for d, _, fs in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def imported_modules(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield ("." * node.level) + (node.module or "")


def test_product_does_not_use_the_oracle():
    for p in files(PKG, (".py",)):
        for m in imported_modules(p):
            assert not m.split(".")[0] == "oracle", (p, m)
        src = open(p).read()
        assert "gea_oracle" not in src and "libgea_oracle" not in src, p
    for p in files(PKG, (".cu", ".cuh", ".h")):
        src = open(p).read()
        assert not re.search(r'#include\s*"[^"]*oracle', src), p
        assert "orc_" not in src, p


def test_oracle_does_not_use_the_product():
    for p in files(ORC, (".py",)):
        for m in imported_modules(p):
            assert not m.startswith("paper_2303_10499_gb300"), (p, m)
    for p in files(ORC, (".c", ".h")):
        for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(p).read()):
            assert inc in ("math.h", "stdint.h", "stdlib.h", "string.h", "stdio.h", "stddef.h"), (p, inc)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without its CUDA library the binding raises; it has nothing to fall
    back on."""
    import pytest
    from paper_2303_10499_gb300 import gea
    monkeypatch.setattr(gea, "_lib", None)
    monkeypatch.setattr(gea, "LIB", str(tmp_path / "libgea.so"))
    with pytest.raises(RuntimeError, match="not built"):
        gea.library()
