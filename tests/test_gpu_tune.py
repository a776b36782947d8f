"""The autotuner and the tuning fields: every tuning gives the same answers bit
for bit; rkr_autotune picks one by timed trials, sets it, and caches it."""

import json

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")

DEFAULT = dict(rc_bn=256, rc_single_first=1, skip_level=0, cand_budget_log2=26,
               latency_ctas_per_sm=0, latency_bulk=0, screen_form=1, rc_seg_min=0,
               split_cat=1, rc_prefix=4)


def _answers(idx, w):
    u, r, _, _ = idx.query_exact(w.Q, w.k)
    a = idx.query_approx(w.Q, w.k, 2.0)
    s = idx.query_approx(w.Q, w.k, 2.0, single=True)
    return [u, r] + [a[key] for key in ("users", "n_low", "n_up", "est", "case", "nc")] + \
        [s[key] for key in ("users", "n_low", "n_up", "est")]


def test_every_tuning_gives_the_same_answers(tmp_path):
    w = synth.make_workload("approx", n=12000, m=2500, d=40, nq=40)
    pos = synth.sample_positions(2, oracle.bucket_sizes(w.m, 5), 40)
    try:
        with rkr.Index(w.U, w.P, tau=64, omega=5, s=40, sample_pos=pos, exact_table=True,
                       floor_rank=40) as idx:
            rkr.rkr_tuning_set(**DEFAULT)
            ref = _answers(idx, w)
            for fields in (dict(rc_bn=128), dict(rc_single_first=0), dict(skip_level=3),
                           dict(skip_level=9), dict(cand_budget_log2=20),
                           dict(latency_ctas_per_sm=2), dict(latency_bulk=1),
                           dict(screen_form=0), dict(screen_form=2), dict(rc_seg_min=2),
                           dict(rc_seg_min=4, rc_single_first=0), dict(split_cat=0),
                           dict(rc_prefix=0), dict(rc_prefix=2)):
                rkr.rkr_tuning_set(**{**DEFAULT, **fields})
                got = _answers(idx, w)
                for a, b in zip(got, ref):
                    assert (a == b).all(), fields
            rkr.rkr_tuning_set(**DEFAULT)
            cache = tmp_path / "tune.jsonl"
            t1, ms1 = idx.autotune(w.Q, w.k, what=7, cache_path=str(cache))
            assert rkr.rkr_tuning_get() == t1 and ms1 > 0
            lines = cache.read_text().splitlines()
            assert len(lines) == 1 and json.loads(lines[0])["rc_bn"] == t1["rc_bn"]
            for a, b in zip(_answers(idx, w), ref):
                assert (a == b).all()
            rkr.rkr_tuning_set(**DEFAULT)
            t2, ms2 = idx.autotune(w.Q, w.k, what=7, cache_path=str(cache))   # from the cache
            assert t2 == t1 and ms2 == pytest.approx(ms1, abs=1e-3)
            assert len(cache.read_text().splitlines()) == 1
    finally:
        rkr.rkr_tuning_set(**DEFAULT)


def test_screen_forms_build_the_same_index():
    # 157 row blocks of 128 users: the last CTA pair has one block past the end
    w = synth.make_workload("approx", n=20000, m=3000, d=72, nq=30)
    pos = synth.sample_positions(4, oracle.bucket_sizes(w.m, 5), 30)
    names = ("fmin", "fmax", "table", "xlo", "xhi", "xgrid")
    ref = None
    try:
        # the split product's two operand layouts (d = 72: K' = 80 gives 4 stages per
        # tile concatenated against 6 in segments)
        for form, cat in ((0, 1), (1, 1), (2, 1), (1, 0), (2, 0)):
            rkr.rkr_tuning_set(**{**DEFAULT, "screen_form": form, "split_cat": cat})
            with rkr.Index(w.U, w.P, tau=48, omega=5, s=30, sample_pos=pos, exact_table=True,
                           floor_rank=40) as idx:
                got = [idx.export(x) for x in names]
                got += list(idx.query_exact(w.Q, w.k)[:2])
                a = idx.query_approx(w.Q, w.k, 2.0)
                got += [a[key] for key in ("users", "n_low", "n_up", "est", "case", "nc")]
            if ref is None:
                ref = got
                continue
            for i, (x, y) in enumerate(zip(got, ref)):
                assert np.array_equal(x, y), (form, cat, i)
    finally:
        rkr.rkr_tuning_set(**DEFAULT)
