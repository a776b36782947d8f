"""rkr_query_approx_single (queries answered one at a time) against the batched
path and the oracle's transcription of Section 4.3.

The one-at-a-time path computes u.q for every user with FP32 warp products and
its own error bound, so it must reach exactly the same bins, bounds, estimates
and answers as rkr_query_approx and as the oracle: bit for bit.  Cases cover
d divisible by 4 (vector loads) and not, a ragged user count, k = n, c = 1, and
a query far outside the item norms (bins rebuilt for a larger range).
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")

KEYS = ("users", "n_low", "n_up", "est", "case", "nc")


def _run(w, tau, omega, s, c, k):
    pos = synth.sample_positions(3, oracle.bucket_sizes(w.m, omega), s)
    with rkr.Index(w.U, w.P, tau=tau, omega=omega, s=s, sample_pos=pos,
                   exact_table=False) as idx:
        one = idx.query_approx(w.Q, k, c, single=True)
        batch = idx.query_approx(w.Q, k, c)
    for key in KEYS:
        assert (one[key] == batch[key]).all(), key
    ora = oracle.build_index(w.U, w.P, tau, omega, s, pos)
    kk = np.broadcast_to(np.asarray(k), (w.Q.shape[0],))
    for q, a in enumerate(oracle.approx_query(ora, w.U, w.Q, kk, c)):
        sl = slice(one["offsets"][q], one["offsets"][q + 1])
        assert (one["users"][sl] == a["users"]).all(), q
        assert (one["n_low"][sl] == a["n_low"]).all(), q
        assert (one["n_up"][sl] == a["n_up"]).all(), q
        assert (one["est"][sl] == a["est"]).all(), q
        assert one["case"][q] == a["case"] and one["nc"][q] == a["nc"], q
    return one


@pytest.mark.parametrize("d", [64, 37])
def test_single_equals_batched_and_oracle(d):
    w = synth.make_workload("approx", n=4097, m=1200, d=d, nq=12)
    _run(w, 60, 4, 40, 2.0, w.k)


def test_single_edge_cases():
    w = synth.make_workload("approx", n=300, m=500, d=24, nq=4)
    _run(w, 20, 3, 25, 1.0, 300)            # k = n, c = 1
    w.Q[1] *= np.float32(50.0)              # far outside the item norms
    _run(w, 20, 3, 25, 2.0, np.array([1, 7, 300, 30], np.int32))


def test_session_graph_answers_equal_the_batch():
    w = synth.make_workload("approx", n=5000, m=1500, d=48, nq=10)
    pos = synth.sample_positions(3, oracle.bucket_sizes(w.m, 4), 40)
    w.Q[7] *= np.float32(40.0)          # beyond the item norms: answered without the graph
    with rkr.Index(w.U, w.P, tau=50, omega=4, s=40, sample_pos=pos, exact_table=False) as idx:
        batch = idx.query_approx(w.Q, w.k, 2.0)
        with rkr.Session(idx, max_k=int(w.k.max()), c=2.0) as sess:
            for rep in range(2):       # the graph is replayed: nothing carries over
                for q in range(w.Q.shape[0]):
                    got = sess.query(w.Q[q], int(w.k[q]))
                    sl = slice(batch["offsets"][q], batch["offsets"][q + 1])
                    for key in ("users", "n_low", "n_up", "est"):
                        assert (got[key] == batch[key][sl]).all(), (q, key)
                    assert got["case"][0] == batch["case"][q] and got["nc"][0] == batch["nc"][q]
            import torch
            qd = torch.from_numpy(w.Q[2]).cuda()      # a device query vector
            got = sess.query(qd, int(w.k[2]))
            sl = slice(batch["offsets"][2], batch["offsets"][3])
            assert (got["users"] == batch["users"][sl]).all()
            with pytest.raises(rkr.RKRError):
                sess.query(w.Q[0], int(w.k.max()) + 1)
            bad = w.Q[0].copy()
            bad[3] = np.nan
            with pytest.raises(rkr.RKRError):
                sess.query(bad, 1)
