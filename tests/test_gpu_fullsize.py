"""Parity at the full workload sizes, on outputs the oracle can compute one by one.

The two exact workloads run at full size on the GPU:
- 500,000 users x 20,000 items x d = 100, 1,024 queries, k = 100;
- 1M x 100k x d = 200, 10,000 queries, with the index parameters the benchmark
  uses (tau 500, omega 10, s 100, exact f-bounds and count tables).

For sampled queries:
- every returned rank equals the oracle's rank of that user (Def. 1);
- the answer is ordered by (rank, user);
- no sampled user outside the answer ranks better than the k-th, or ties it
  with a smaller index (Def. 2).

For the 1M x 100k index, the pre-processing of sampled users (f_min, f_max and
the Eq. 1 numerators) is compared bit for bit with the oracle's index of those
users.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")


def _check_sampled(w, users, ranks, off, queries, rng, n_out):
    for q in queries:
        sl = slice(off[q], off[q + 1])
        u, r = users[sl], ranks[sl]
        assert len(u) == w.k[q]
        assert (r == oracle.ranks(w.U[u], w.P, w.Q[q:q + 1])[:, 0]).all(), q
        key = r.astype(np.int64) * (1 << 32) + u.astype(np.int64)
        assert (np.diff(key) > 0).all(), q
        kth = int(r.max())
        last = int(u[r == kth].max())
        others = np.setdiff1d(rng.choice(w.n, size=n_out, replace=False), u)
        ro = oracle.ranks(w.U[others], w.P, w.Q[q:q + 1])[:, 0]
        assert ((ro > kth) | ((ro == kth) & (others > last))).all(), q


def test_exact_batched_workload_full_size():
    w = synth.make_workload("exact_batched")
    rng = np.random.default_rng(21)
    with rkr.Index(w.U, w.P, exact_table=True) as idx:
        users, ranks, off, _ = idx.query_exact(w.Q, w.k)
    queries = np.concatenate([rng.choice(512, 8, replace=False),
                              512 + rng.choice(512, 8, replace=False)])  # from P and fresh
    _check_sampled(w, users, ranks, off, queries, rng, n_out=1000)


def test_approx_workload_full_size_exact_answers_and_index():
    w = synth.make_workload("approx")
    sizes = oracle.bucket_sizes(w.m, w.omega)
    pos = synth.sample_positions(w.seed, sizes, w.s)
    rng = np.random.default_rng(22)
    with rkr.Index(w.U, w.P, tau=w.tau, omega=w.omega, s=w.s, fbounds="exact",
                   exact_table=True, sample_pos=pos) as idx:
        users, ranks, off, _ = idx.query_exact(w.Q, w.k)
        fmin, fmax = idx.export("fmin"), idx.export("fmax")
        table = idx.export("table")
    _check_sampled(w, users, ranks, off, rng.choice(w.Q.shape[0], 12, replace=False), rng,
                   n_out=500)
    sample = np.sort(rng.choice(w.n, size=128, replace=False))
    ora = oracle.build_index(w.U[sample], w.P, w.tau, w.omega, w.s, pos)
    assert (fmin[sample] == ora["fmin"]).all()
    assert (fmax[sample] == ora["fmax"]).all()
    assert (table[sample] == ora["N"]).all()


def test_approx_workload_full_size_approximate_answers():
    """The c-approximate query path at full size (1M x 100k x 200, tau 500, omega 10,
    s 100, c = 2, all 10,000 queries in one batch) against the oracle's own full
    index.  The oracle builds that index with the footnote's Cauchy-Schwarz
    f-bounds (one FP64 norm per row) so that its full Alg. 1 table of 1M users is
    affordable on the host; the GPU index is built the same way.  The query steps
    (the u.q screen, the bounds lookup, R_low_k and R_up_k, Case A/B and the
    interpolation) do not depend on how f_min and f_max were found.  For sampled
    queries users, numerators, FP64 estimates, case and |U_c| must match bit for bit."""
    w = synth.make_workload("approx")
    sizes = oracle.bucket_sizes(w.m, w.omega)
    pos = synth.sample_positions(w.seed, sizes, w.s)
    rng = np.random.default_rng(23)
    with rkr.Index(w.U, w.P, tau=w.tau, omega=w.omega, s=w.s, fbounds="cs",
                   exact_table=False, sample_pos=pos) as idx:
        got = idx.query_approx(w.Q, w.k, 2.0)
    ora = oracle.build_index(w.U, w.P, w.tau, w.omega, w.s, pos, fbounds="cs")
    queries = np.sort(rng.choice(w.Q.shape[0], 6, replace=False))
    theta = oracle.scores(w.U, w.Q[queries])
    for i, q in enumerate(queries):
        want = oracle.approx_query_one(ora, theta[:, i], int(w.k[q]), 2.0)
        sl = slice(got["offsets"][q], got["offsets"][q + 1])
        assert (got["users"][sl] == want["users"]).all(), q
        assert (got["n_low"][sl] == want["n_low"]).all(), q
        assert (got["n_up"][sl] == want["n_up"]).all(), q
        assert (got["est"][sl] == want["est"]).all(), q
        assert got["case"][q] == want["case"] and got["nc"][q] == want["nc"], q
