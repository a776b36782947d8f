"""Users split into parts on one GPU (the parts run one after another in this
process), merged by the host merge: the answer equals one index over all users,
bit for bit, for exact and c-approximate queries.  Each part builds its own index
from its rows with the same items, build parameters and sample positions."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")
from paper_2504_13446_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("parts", [2, 3])
def test_parts_merge_equals_one_index(parts):
    w = synth.make_workload("approx", n=20_001, m=3000, d=48, nq=24)
    w.k = np.resize(np.array([1, 10, 50, 100, 400], np.int32), w.Q.shape[0])
    tau, omega, s, c = 80, 6, 50, 2.0
    pos = synth.sample_positions(8, oracle.bucket_sizes(w.m, omega), s)
    kw = dict(tau=tau, omega=omega, s=s, sample_pos=pos, exact_table=True)
    with rkr.Index(w.U, w.P, **kw) as whole:
        want_a = whole.query_approx(w.Q, w.k, c)
        want_u, want_r, _, _ = whole.query_exact(w.Q, w.k)
    ex_parts, ap_parts = [], []
    for p in range(parts):
        a, b = shard.shard_range(w.n, parts, p)
        kl = np.minimum(w.k, b - a).astype(np.int32)
        with rkr.Index(w.U[a:b], w.P, **kw) as idx:
            u, r, off, _ = idx.query_exact(w.Q, kl)
            ex_parts.append({"offsets": off, "users": u.astype(np.int64) + a, "ranks": r})
            ap_parts.append(idx.query_approx_candidates(w.Q, kl, user_offset=a))
    offs, cat = shard.concat_parts(ex_parts, ("users", "ranks"))
    got_u, got_r, _ = rkr.rkr_merge_exact(w.k, offs, cat["users"], cat["ranks"])
    assert (got_u == want_u).all() and (got_r == want_r).all()
    offs, cat = shard.concat_parts(ap_parts, ("users", "n_low", "n_up", "est"))
    got = rkr.rkr_merge_approx(w.k, c, s, offs, cat["users"], cat["n_low"], cat["n_up"],
                               cat["est"])
    for key in ("users", "n_low", "n_up", "est", "case", "nc"):
        assert (got[key] == want_a[key]).all(), key
