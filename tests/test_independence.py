"""The oracle and the CUDA path share no code, and the product path has no CPU
fallback (CPU only).

- Nothing in the package (Python binding, CUDA sources, headers) imports,
  includes or loads anything under oracle/; nothing under oracle/ includes
  the library's headers or imports the package.  Only the seeded input
  generators (paper_1601_04641_gb300/inputs.py, which holds none of the
  method's arithmetic) serve both sides, through the tests.
- With libgpcn.so missing, loading the binding and creating a handle raise
  instead of computing anything elsewhere."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1601_04641_gb300")


def sources(top, exts):
    for d, _, files in os.walk(top):
        if "__pycache__" in d:
            continue
        for fn in files:
            if fn.endswith(exts):
                yield os.path.join(d, fn)


def test_package_never_reaches_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b|#\s*include\s*[<\"][^>\"]*oracle)|"
                     r"gp_oracle|liboracle|oracle[/\\]", re.M)
    hits = []
    for path in sources(PKG, (".py", ".cu", ".cuh", ".h", ".cpp", ".c")):
        text = open(path, encoding="utf-8").read()
        hits += ["%s: %s" % (os.path.relpath(path, ROOT), m.group(0).strip()) for m in pat.finditer(text)]
    assert not hits, hits


def test_oracle_never_reaches_the_package():
    pat = re.compile(r"^\s*(import\s+paper_1601_04641_gb300\b|from\s+paper_1601_04641_gb300\b|"
                     r"#\s*include\s*\"[^\"]*\")|libgpcn|csrc", re.M)
    hits = []
    for path in sources(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        text = open(path, encoding="utf-8").read()
        hits += ["%s: %s" % (os.path.relpath(path, ROOT), m.group(0).strip()) for m in pat.finditer(text)]
    assert not hits, hits


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1601_04641_gb300 import _native as N
    from paper_1601_04641_gb300 import solver
    monkeypatch.setattr(N, "LIB_PATH", str(tmp_path / "libgpcn.so"))
    monkeypatch.setattr(N, "_lib", None)
    with pytest.raises(RuntimeError, match="no fallback"):
        N.load()
    with pytest.raises(RuntimeError, match="no fallback"):
        solver.GP((8, 8, 8), (0.1, 0.1, 0.1), 1e-3, (1.0, 1.0, 1.0), 1.0, "f64", "complex")
