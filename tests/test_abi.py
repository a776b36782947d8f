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
    monkeypatch.setattr(pkg.buildlib, "lib_path", lambda variant="single_gpu":
                        str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(RuntimeError):
        pkg.load()


def test_replica_build_exports_every_symbol_and_names_itself():
    from paper_2504_13446_gb300 import buildlib
    single = ctypes.CDLL(buildlib.build())
    replica = ctypes.CDLL(buildlib.build(variant="replica"))
    for name in _declared():
        assert hasattr(replica, name), name
    for lib in (single, replica):
        lib.rkr_version.restype = ctypes.c_char_p
    assert b"single-GPU build" in single.rkr_version()
    assert b"replica build" in replica.rkr_version()


def test_cluster_multicast_stays_out_of_the_replica_build():
    """Only tc_pair.cuh names a multicast TMA load or commit, and no translation
    unit of the replica build (the one a rank of a multi-GPU job loads) includes it."""
    from paper_2504_13446_gb300 import buildlib
    csrc = buildlib.CSRC
    for f in sorted(os.listdir(csrc)):
        text = open(os.path.join(csrc, f)).read()
        if f != "tc_pair.cuh":
            assert ".multicast::cluster" not in text, f
    uses_pair = 0
    for src in buildlib._sources():
        assert "tc_pair.cuh" not in buildlib.included_headers(src, "replica"), src
        uses_pair += "tc_pair.cuh" in buildlib.included_headers(src, "single_gpu")
    assert uses_pair >= 1


def test_variant_selection(monkeypatch):
    from paper_2504_13446_gb300 import buildlib
    monkeypatch.delenv("RKR_LIB_VARIANT", raising=False)
    assert buildlib.selected_variant() == "single_gpu"
    monkeypatch.setenv("RKR_LIB_VARIANT", "replica")
    assert buildlib.lib_path(buildlib.selected_variant()).endswith("librkr_replica.so")
    monkeypatch.setenv("RKR_LIB_VARIANT", "bogus")
    with pytest.raises(RuntimeError):
        buildlib.selected_variant()


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2504_13446_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_tuning_fields_are_validated_without_a_gpu():
    import paper_2504_13446_gb300 as pkg
    pkg.buildlib.build()
    before = pkg.rkr_tuning_get()
    try:
        for bad in (dict(rc_bn=64), dict(rc_single_first=2), dict(skip_level=31),
                    dict(cand_budget_log2=19), dict(latency_ctas_per_sm=-1),
                    dict(latency_bulk=2), dict(screen_form=3), dict(rc_seg_min=1),
                    dict(rc_seg_min=33), dict(split_cat=2), dict(rc_prefix=1),
                    dict(rc_prefix=65), dict(rc_prefix=-1)):
            with pytest.raises(pkg.RKRError):
                pkg.rkr_tuning_set(**bad)
        pkg.rkr_tuning_set(rc_bn=128)
        assert pkg.rkr_tuning_get()["rc_bn"] == 128
    finally:
        pkg.rkr_tuning_set(**before)
