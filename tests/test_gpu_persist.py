"""rkr_index_save / rkr_index_load and rkr_pruner_save / rkr_pruner_load.

A saved and reloaded index answers exact and c-approximate queries bit for bit
like the index it was saved from, and exports the same arrays; a corrupted or
truncated file is refused with RKR_EINVAL.  A reloaded pruner predicts exactly
as the saved one.
"""

import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")

EINVAL = 1


def _index_and_queries(exact_table=True):
    w = synth.make_workload("approx", n=3000, m=1500, d=40, nq=20)
    pos = synth.sample_positions(1, oracle.bucket_sizes(w.m, 5), 30)
    idx = rkr.Index(w.U, w.P, tau=40, omega=5, s=30, sample_pos=pos, exact_table=exact_table)
    return w, idx


@pytest.mark.parametrize("exact_table", [True, False, 2])
def test_round_trip_answers_bit_for_bit(tmp_path, exact_table):
    w, idx = _index_and_queries(exact_table)
    path = str(tmp_path / "index.rkr")
    with idx:
        a0 = idx.query_approx(w.Q, w.k, 2.0)
        e0 = idx.query_exact(w.Q, w.k) if exact_table else None
        names = ("perm", "fmin", "fmax", "table", "samples", "pnorm")
        if exact_table == 2:
            names += ("dlo", "dhi", "dgrid")
        ex0 = {n: idx.export(n) for n in names}
        idx.save(path)
    with rkr.Index.load(path) as idx2:
        assert idx2.info == idx.info
        a1 = idx2.query_approx(w.Q, w.k, 2.0)
        for key in ("users", "n_low", "n_up", "est", "case", "nc"):
            assert (a1[key] == a0[key]).all(), key
        if exact_table:
            e1 = idx2.query_exact(w.Q, w.k)
            assert (e1[0] == e0[0]).all() and (e1[1] == e0[1]).all()
        for n, v in ex0.items():
            assert (idx2.export(n) == v).all(), n


def test_corrupt_and_truncated_files_are_refused(tmp_path):
    w, idx = _index_and_queries(True)
    path = str(tmp_path / "index.rkr")
    with idx:
        idx.save(path)
    raw = open(path, "rb").read()
    bad = bytearray(raw)
    bad[len(raw) // 2] ^= 0x40
    (tmp_path / "bad.rkr").write_bytes(bytes(bad))
    (tmp_path / "short.rkr").write_bytes(raw[: len(raw) // 3])
    (tmp_path / "junk.rkr").write_bytes(b"not an index at all")
    for name in ("bad.rkr", "short.rkr", "junk.rkr", "missing.rkr"):
        with pytest.raises(rkr.RKRError) as e:
            rkr.Index.load(str(tmp_path / name))
        assert e.value.status == EINVAL, name


def test_pruner_round_trip(tmp_path):
    rng = np.random.default_rng(4)
    net = rkr.Pruner(65, 64, seed=9)
    X = rng.standard_normal((500, 65)).astype(np.float32)
    t = rng.standard_normal(500).astype(np.float32)
    net.train(X, t, rng.standard_normal(500).astype(np.float32), epochs=1, batch=128)
    path = str(tmp_path / "pruner.rkr")
    net.save(path)
    net2 = rkr.Pruner.load(path)
    assert (net2.forward(X, t) == net.forward(X, t)).all()
    assert (net2.get_params() == net.get_params()).all()
    raw = bytearray(open(path, "rb").read())
    raw[40] ^= 1
    (tmp_path / "bad.rkr").write_bytes(bytes(raw))
    with pytest.raises(rkr.RKRError):
        rkr.Pruner.load(str(tmp_path / "bad.rkr"))
