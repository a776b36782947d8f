"""Device memory kept for reuse: an index built into recycled pool memory, and
one built after the pool was trimmed, answer exactly like the first."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")


def _answers(w):
    idx = rkr.Index(w.U, w.P, tau=w.tau, omega=w.omega, s=w.s, exact_table=True)
    try:
        eu, er, _, _ = idx.query_exact(w.Q, w.k)
        a = idx.query_approx(w.Q, w.k, 2.0)
        return eu, er, a["users"]
    finally:
        idx.close()


def test_rebuilds_from_recycled_and_trimmed_memory_agree():
    w = synth.make_workload("approx", n=6000, m=3000, nq=40)
    first = _answers(w)
    again = _answers(w)                 # arrays come back from the pool
    rkr.rkr_release_cached_memory()
    trimmed = _answers(w)               # and from fresh memory after the trim
    for x, y, z in zip(first, again, trimmed):
        assert (x == y).all() and (x == z).all()
