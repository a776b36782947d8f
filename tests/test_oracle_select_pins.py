"""Pins of the oracle's per-query drivers.

select_exact (Def. 2 with the (rank, index) tie reading) is compared with a
brute-force sort of (rank, user) pairs, with heavy ties and with user subsets.
approx_query (Section 4.3 over a batch) is compared with approx_query_one on
u.q values formed one pair at a time by the oracle's scalar dot product, and
its subset answers must lie inside the subset.
"""

import numpy as np

import oracle
import synth


def test_select_exact_is_the_k_smallest_rank_index_pairs():
    rng = np.random.default_rng(3)
    for trial in range(50):
        n = int(rng.integers(1, 40))
        col = rng.integers(1, 6, size=n).astype(np.int32)   # many ties
        k = int(rng.integers(1, n + 1))
        users, ranks = oracle.select_exact(col, k)
        want = sorted((int(col[u]), u) for u in range(n))[:k]
        assert [(int(r), int(u)) for r, u in zip(ranks, users)] == want
        sub = np.sort(rng.choice(n, size=int(rng.integers(1, n + 1)), replace=False))
        ks = int(rng.integers(1, len(sub) + 1))
        users, ranks = oracle.select_exact(col[sub], ks, sub)
        want = sorted((int(col[u]), int(u)) for u in sub)[:ks]
        assert [(int(r), int(u)) for r, u in zip(ranks, users)] == want


def test_approx_query_matches_one_query_at_a_time():
    w = synth.make_workload("approx", n=60, m=300, nq=5, d=8)
    tau, omega, s = 12, 3, 20
    pos = synth.sample_positions(1, oracle.bucket_sizes(w.m, omega), s)
    idx = oracle.build_index(w.U, w.P, tau, omega, s, pos)
    k = np.array([1, 3, 5, 10, 60])
    batch = oracle.approx_query(idx, w.U, w.Q, k, 2.0)
    for q in range(w.Q.shape[0]):
        theta = np.array([oracle.dot(w.U[u], w.Q[q]) for u in range(w.n)])
        one = oracle.approx_query_one(idx, theta, int(k[q]), 2.0)
        assert (batch[q]["users"] == one["users"]).all()
        assert (batch[q]["est"] == one["est"]).all()
    rng = np.random.default_rng(4)
    subsets = [np.sort(rng.choice(w.n, size=30, replace=False)) for _ in range(w.Q.shape[0])]
    ks = np.minimum(k, 30)
    sub = oracle.approx_query(idx, w.U, w.Q, ks, 2.0, subsets=subsets)
    for q in range(w.Q.shape[0]):
        assert len(sub[q]["users"]) == ks[q]
        assert np.isin(sub[q]["users"], subsets[q]).all()
