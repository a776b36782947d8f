"""Exact ranks of arbitrary pairs, and the learned pruner on exact ranks from the GPU path.

rkr_rank_pairs is compared with the oracle's ranks bit for bit.  The pruner is
trained on ranks that rkr_rank_pairs produces for training queries, then cuts
the exact path's candidates of other queries: without the fallback every rank
it returns is the oracle's, it recounts fewer candidates and its recall is
bounded below; with the exact fallback (cut candidates whose rank lower bound
can still reach the k-th rank are recounted) the answer equals
rkr_query_exact's, users and ranks.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")


def test_rank_pairs_match_oracle():
    w = synth.make_workload("exact_small", n=3000, m=2500, nq=12)
    rng = np.random.default_rng(5)
    gpu = rkr.Index(w.U, w.P, tau=32, omega=5, s=25, exact_table=True, floor_rank=60)
    pu = rng.integers(0, w.n, size=5000).astype(np.int32)
    pq = rng.integers(0, 12, size=5000).astype(np.int32)
    got = gpu.rank_pairs(w.Q, pu, pq)
    R = oracle.ranks(w.U, w.P, w.Q)
    assert (got == R[pu, pq]).all()
    with pytest.raises(rkr.RKRError):
        gpu.rank_pairs(w.Q, np.array([w.n], np.int32), np.array([0], np.int32))


def test_learned_cut_returns_exact_ranks_with_high_recall():
    w = synth.make_workload("approx", n=20000, m=4000, nq=96)
    rng = np.random.default_rng(11)
    # a low floor rank puts the tail lists' end at rank ~32, so most candidates of
    # the k = 50 and k = 100 queries need a recount over P: the set the cut acts on
    gpu = rkr.Index(w.U, w.P, tau=w.tau, omega=w.omega, s=w.s, exact_table=True, floor_rank=32)
    Rp = (rng.standard_normal((64, w.d)) / np.sqrt(w.d)).astype(np.float32)
    train_q, eval_q = w.Q[:64], w.Q[64:]
    k_eval = w.k[64:]
    # training pairs: every training query against random users and its 400 best users
    users_t, _, _, _ = gpu.query_exact(train_q, 400)
    pu = np.concatenate([rng.integers(0, w.n, size=64 * 200), users_t]).astype(np.int32)
    pq = np.concatenate([np.repeat(np.arange(64), 200), np.repeat(np.arange(64), 400)])
    pq = pq.astype(np.int32)
    r = gpu.rank_pairs(train_q, pu, pq)
    X, t = gpu.pair_features(Rp, train_q, pu, pq)
    net = rkr.Pruner(65, 256, seed=2)
    net.train(X, t, np.log(r).astype(np.float32), epochs=30, batch=512, lr=2e-3, seed=3)
    # evaluation: the cut against the plain exact path
    plain_u, plain_r, off, plain_st = gpu.query_exact(eval_q, k_eval)
    R = oracle.ranks(w.U, w.P, eval_q)
    qid = np.repeat(np.arange(len(eval_q)), np.diff(off))
    # the plain cut: ranks exact, recall judged against the exact query
    keep = 2 * k_eval          # recount at most 2k candidates per query
    lu, lr, loff, st = gpu.query_exact_learned(net, Rp, eval_q, k_eval, keep, certify=False)
    assert (loff == off).all()
    assert (lr == R[lu, qid]).all()                  # ranks returned are exact
    hits = sum(int(np.sum(lr[off[q]:off[q + 1]] <= plain_r[off[q]:off[q + 1]].max()))
               for q in range(len(eval_q)))
    recall = hits / float(off[-1])
    print(f"learned cut: keep 2k, recall {recall:.4f}, {st.candidates} candidates instead of "
          f"{plain_st.candidates}, recounted {st.recounted} instead of {plain_st.recounted}")
    assert st.candidates < plain_st.candidates and st.recounted < plain_st.recounted
    assert recall >= 0.9
    # with the exact fallback: the exact answer, whatever the cut
    for factor in (2, 1):
        lu, lr, loff, st = gpu.query_exact_learned(net, Rp, eval_q, k_eval, factor * k_eval,
                                                   certify=True)
        assert (loff == off).all()
        assert (lu == plain_u).all() and (lr == plain_r).all()
        print(f"certified cut: keep {factor}k, {st.learned_revived} candidates revived")
    # keep as an array, one per query: a keep no smaller than any query's candidate
    # count cuts nothing, so the answer is the plain exact one
    big = np.full(len(eval_q), w.n, np.int32)
    bu, br, boff, bst = gpu.query_exact_learned(net, Rp, eval_q, k_eval, big)
    assert (bu == plain_u).all() and (br == plain_r).all() and (boff == off).all()
    assert bst.candidates == plain_st.candidates
    # and keep below k is rejected
    small = k_eval.copy()
    small[3] -= 1
    with pytest.raises(rkr.RKRError):
        gpu.query_exact_learned(net, Rp, eval_q, k_eval, small)


def test_pruner_tables_match_the_network_and_cut_exactly():
    """rkr_pruner_invert tabulates the network per user on a grid of t; each table
    row never increases (the network is monotone in t by construction), its
    entries are the network's outputs at the grid points, and a learned query
    that predicts by table lookup returns exact ranks, and with the fallback the
    exact answer.  New weights drop the tables."""
    w = synth.make_workload("approx", n=8000, m=3000, nq=64)
    rng = np.random.default_rng(21)
    gpu = rkr.Index(w.U, w.P, tau=w.tau, omega=w.omega, s=w.s, exact_table=True, floor_rank=32)
    Rp = (rng.standard_normal((64, w.d)) / np.sqrt(w.d)).astype(np.float32)
    train_q, eval_q, k_eval = w.Q[:32], w.Q[32:], w.k[32:]
    users_t, _, _, _ = gpu.query_exact(train_q, 200)
    pu = np.concatenate([rng.integers(0, w.n, size=32 * 200), users_t]).astype(np.int32)
    pq = np.concatenate([np.repeat(np.arange(32), 200), np.repeat(np.arange(32), 200)])
    pq = pq.astype(np.int32)
    r = gpu.rank_pairs(train_q, pu, pq)
    X, t = gpu.pair_features(Rp, train_q, pu, pq)
    net = rkr.Pruner(65, 256, seed=4)
    net.train(X, t, np.log(r).astype(np.float32), epochs=10, batch=512, lr=2e-3, seed=5)
    G = 32
    net.invert(gpu, Rp, G)
    tab, grid = net.table(w.n, G)
    assert np.isfinite(tab).all() and (np.diff(tab, axis=1) <= 0).all()
    fmin, fmax = gpu.export("fmin"), gpu.export("fmax")
    unorm = np.linalg.norm(w.U.astype(np.float64), axis=1)
    assert np.allclose(grid[:, 0], fmin / unorm, rtol=1e-5, atol=1e-6)
    assert np.allclose(grid[:, 0] + (G - 1) * grid[:, 1].astype(np.float64), fmax / unorm,
                       rtol=1e-4, atol=1e-5)
    # entries are the network's outputs at the grid points of sampled users
    su = rng.choice(w.n, 50, replace=False).astype(np.int32)
    Xs, _ = gpu.pair_features(Rp, eval_q, su, np.zeros(len(su), np.int32))
    tg = (grid[su, 0][:, None].astype(np.float64)
          + np.arange(G)[None, :] * grid[su, 1][:, None].astype(np.float64)).astype(np.float32)
    y = net.forward(np.repeat(Xs, G, axis=0), tg.reshape(-1)).reshape(len(su), G)
    assert np.allclose(y, tab[su], rtol=1e-4, atol=1e-4), np.abs(y - tab[su]).max()
    # learned queries by table lookup
    plain_u, plain_r, off, _ = gpu.query_exact(eval_q, k_eval)
    R = oracle.ranks(w.U, w.P, eval_q)
    qid = np.repeat(np.arange(len(eval_q)), np.diff(off))
    lu, lr, loff, st = gpu.query_exact_learned(net, Rp, eval_q, k_eval, 2 * k_eval,
                                               certify=False)
    assert (loff == off).all() and (lr == R[lu, qid]).all()
    cu, cr, coff, _ = gpu.query_exact_learned(net, Rp, eval_q, k_eval, k_eval, certify=True)
    assert (cu == plain_u).all() and (cr == plain_r).all()
    # another projection does not match the tables: the network predicts, same answer
    Rq = Rp * np.float32(1.5)
    cu2, cr2, _, _ = gpu.query_exact_learned(net, Rq, eval_q, k_eval, k_eval, certify=True)
    assert (cu2 == plain_u).all() and (cr2 == plain_r).all()
    # new weights drop the tables; G = 0 is accepted with or without them
    net.set_params(net.get_params())
    with pytest.raises(rkr.RKRError):
        net.table(w.n, G)
    net.invert(gpu, Rp, 0)
    with pytest.raises(rkr.RKRError):
        net.invert(gpu, Rp, 1)
