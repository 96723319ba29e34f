"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and exports every
function that include/hisq.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hisq_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2306_01098_gb300 import build, hisq
    build.build()
    lib = ctypes.CDLL(build.LIB)
    decl = declared_functions()
    assert len(decl) >= 15
    missing = [n for n in decl if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the whole ABI
    assert set(decl) <= set(hisq.exported_symbols())


def test_binding_raises_without_library(monkeypatch, tmp_path):
    from paper_2306_01098_gb300 import hisq
    monkeypatch.setattr(hisq, "LIBPATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(hisq, "_lib", None)
    with pytest.raises(RuntimeError):
        hisq.lib()
