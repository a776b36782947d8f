"""Seeded input generators (no method arithmetic): shapes, determinism and the
disjointness of the extra queries the learned part trains and calibrates on."""

import numpy as np

import synth


def test_disjoint_queries_avoid_the_workload_queries_and_repeat_with_the_seed():
    w = synth.make_workload("approx", n=500, m=4000, nq=300)
    Q1, idx1, k1 = synth.disjoint_queries(w, 250, seed=8)
    Q2, idx2, k2 = synth.disjoint_queries(w, 250, seed=8)
    assert (idx1 == idx2).all() and (Q1 == Q2).all() and (k1 == k2).all()
    assert len(np.unique(idx1)) == 250
    assert not np.isin(idx1, w.query_from_P).any()
    assert (Q1 == w.P[idx1]).all()
    assert set(np.unique(k1)) <= {10, 50, 100}
    _, idx3, _ = synth.disjoint_queries(w, 250, seed=9)
    assert not (idx3 == idx1).all()


def test_workloads_have_the_stated_shapes():
    w = synth.make_workload("exact_batched", n=1000, m=300, nq=10)
    assert w.U.shape == (1000, 100) and w.P.shape == (300, 100) and w.Q.shape == (10, 100)
    assert (w.query_from_P[:5] >= 0).all() and (w.query_from_P[5:] == -1).all()
    assert w.U.dtype == np.float32 and (w.k == 100).all()


def test_uneven_subsets_as_blocks_ids_and_bitmaps_agree():
    import numpy as np
    from synth import make_workload
    w = make_workload("uneven", n=5000, m=300, d=16, nq=6)
    bm = w.subset_bitmaps()
    assert bm.shape == (6, (5000 + 31) // 32)
    for q, ids in enumerate(w.subsets):
        bits = np.unpackbits(bm[q].view(np.uint8), bitorder="little")[:5000]
        assert (np.nonzero(bits)[0] == ids).all()
        assert w.k[q] <= len(ids)
        assert not np.unpackbits(bm[q].view(np.uint8), bitorder="little")[5000:].any()
