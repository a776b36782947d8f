"""The C ABI library loads and exports every entry point include/rkr.h declares (no GPU needed)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rkr_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rkr_build", "rkr_query_exact", "rkr_query_approx", "rkr_index_free",
                 "rkr_last_error"):
        assert must in names


def test_library_builds_and_exports_every_symbol():
    from paper_2504_13446_gb300 import buildlib
    lib_path = buildlib.build()
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    import paper_2504_13446_gb300 as pkg
    monkeypatch.setattr(pkg.buildlib, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(RuntimeError):
        pkg.load()


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2504_13446_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f
