"""Per-query user subsets and per-query k (the uneven batch recipe at reduced size).

Exact answers (users, ranks) and the c-approximate outputs are compared bit for
bit with the FP64 oracle run on the same subsets: ranks are over all of P
(Def. 1); the k smallest and the Section 4.3 quantities are over the subset.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")


def _check(U, P, Q, k, subsets, tau, omega, s, c):
    pos = synth.sample_positions(7, oracle.bucket_sizes(P.shape[0], omega), s)
    gpu = rkr.Index(U, P, tau=tau, omega=omega, s=s, sample_pos=pos, exact_table=True)
    users, ranks, off, _ = gpu.query_exact(Q, k, subsets=subsets)
    want = oracle.exact_query(U, P, Q, k, subsets=subsets)
    for q, (wu, wr) in enumerate(want):
        assert (users[off[q]:off[q + 1]] == wu).all() and (ranks[off[q]:off[q + 1]] == wr).all(), q
    ora = oracle.build_index(U, P, tau, omega, s, pos)
    out = gpu.query_approx(Q, k, c, subsets=subsets)
    for q, w in enumerate(oracle.approx_query(ora, U, Q, k, c, subsets=subsets)):
        sl = slice(out["offsets"][q], out["offsets"][q + 1])
        assert out["case"][q] == w["case"] and out["nc"][q] == w["nc"], q
        assert (out["users"][sl] == w["users"]).all(), q
        assert (out["est"][sl] == w["est"]).all(), q


def test_uneven_block_subsets():
    w = synth.make_workload("uneven", n=12000, m=3000, d=128, nq=24)
    _check(w.U, w.P, w.Q, w.k, w.subsets, 48, 6, 40, 2.0)


def test_arbitrary_subsets_and_edge_sizes():
    rng = np.random.default_rng(3)
    w = synth.make_workload("exact_small", n=3000, m=2500, nq=20)
    subsets = []
    for q in range(20):
        size = [1, 2, 50, 3000, 700][q % 5]
        subsets.append(rng.choice(3000, size=size, replace=False).astype(np.int32))
    k = np.array([min(len(s_), kk) for s_, kk in zip(subsets, [1, 1, 17, 200, 64] * 4)],
                 dtype=np.int32)
    _check(w.U, w.P, w.Q, k, subsets, 32, 5, 25, 1.5)


def test_subset_validation():
    rng = np.random.default_rng(4)
    w = synth.make_workload("exact_small", n=500, m=400, nq=3)
    gpu = rkr.Index(w.U, w.P, tau=16, omega=4, s=10, exact_table=True)
    with pytest.raises(rkr.RKRError):   # k above the subset size
        gpu.query_exact(w.Q, 5, subsets=[np.arange(4, dtype=np.int32)] * 3)
    with pytest.raises(rkr.RKRError):   # user id out of range
        gpu.query_exact(w.Q, 1, subsets=[np.array([500], np.int32)] * 3)
    users, ranks, off, _ = gpu.query_exact(w.Q, 1, subsets=[np.array([7], np.int32)] * 3)
    assert (users == 7).all()


def test_bitmap_subsets_equal_id_subsets():
    w = synth.make_workload("uneven", n=9001, m=2000, d=64, nq=12)
    gpu = rkr.Index(w.U, w.P, tau=40, omega=4, s=30, exact_table=True)
    bm = w.subset_bitmaps()
    u1, r1, o1, _ = gpu.query_exact(w.Q, w.k, subsets=w.subsets)
    u2, r2, o2, _ = gpu.query_exact(w.Q, w.k, member=bm)
    assert (u1 == u2).all() and (r1 == r2).all()
    a1 = gpu.query_approx(w.Q, w.k, 2.0, subsets=w.subsets)
    a2 = gpu.query_approx(w.Q, w.k, 2.0, member=bm)
    for key in ("users", "n_low", "n_up", "est", "case", "nc"):
        assert (a1[key] == a2[key]).all(), key
    bad = bm.copy()
    bad[0, -1] |= np.uint32(1 << 31)          # a bit beyond n
    with pytest.raises(rkr.RKRError):
        gpu.query_exact(w.Q, w.k, member=bad)
    with pytest.raises(rkr.RKRError):         # wrong row width
        gpu.query_exact(w.Q, w.k, member=bm[:, :-1])
