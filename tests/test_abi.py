"""The C-ABI library loads on a machine without a GPU and exports every
entry point that include/famst.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "famst.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(famst_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    from paper_2507_14261_gb300 import _build_lib
    path = _build_lib.build()
    L = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 14
    missing = [nm for nm in names if not hasattr(L, nm)]
    assert not missing, missing


def test_error_strings_without_gpu():
    import paper_2507_14261_gb300 as P
    L = P.lib()
    for code in range(0, -10, -1):
        s = L.famst_error_string(code)
        assert s and s != b"unknown status"
    assert L.famst_error_string(-99) == b"unknown status"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2507_14261_gb300.famst as F
    monkeypatch.setattr(F, "_LIB", None)
    monkeypatch.setattr(F._build_lib, "lib_path", lambda: str(tmp_path / "missing.so"))
    import pytest
    with pytest.raises(RuntimeError, match="not built"):
        F.lib()
