"""The bench's approximate-quality report against the oracle's metric code.

bench.approx_quality works from the exact ranks of the returned users and the
exact answer's ranks; oracle.quality works from a full column of exact ranks.
On random rank columns with ties, both must give the same accuracy, overall
ratio, recall and c-bound violations (Def. 3 and the criteria of Section 5).
"""

import numpy as np
import pytest

import bench
import oracle


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bench_quality_equals_oracle_quality(seed):
    rng = np.random.default_rng(seed)
    n, nq, c = 300, 12, 2.0
    ks = rng.integers(1, 40, size=nq)
    off = np.concatenate([[0], np.cumsum(ks)])
    ranks_c, best = [], []
    want = []
    for q in range(nq):
        col = rng.integers(1, 60, size=n)          # exact ranks of every user (ties)
        k = int(ks[q])
        ret = rng.choice(n, size=k, replace=False)  # some returned set
        ranks_c.append(col[ret])
        best.append(np.sort(col)[:k])
        want.append(oracle.quality(col, ret, k, c))
    got = bench.approx_quality(np.concatenate(ranks_c), off, np.concatenate(best), c)
    assert got["queries"] == nq
    assert got["accuracy"] == pytest.approx(np.mean([w["accuracy"] for w in want]))
    assert got["overall_ratio"] == pytest.approx(np.mean([w["overall_ratio"] for w in want]))
    assert got["recall_at_k"] == pytest.approx(np.mean([w["recall"] for w in want]))
    assert got["c_bound_violations"] == sum(w["violations"] for w in want)


def test_exact_answer_scores_perfectly():
    best = np.array([1, 1, 2, 5, 3, 3, 9], dtype=np.int64)
    off = np.array([0, 4, 7])
    ranks_c = np.array([5, 2, 1, 1, 9, 3, 3])   # the same users, in another order
    got = bench.approx_quality(ranks_c, off, best, 2.0)
    assert got["accuracy"] == 1.0 and got["overall_ratio"] == 1.0
    assert got["recall_at_k"] == 1.0 and got["c_bound_violations"] == 0


def test_every_bench_case_has_its_function():
    for name in ("bench_ours", "bench_learned", "bench_latency", "bench_sweep", "bench_uneven",
                 "bench_reference", "learned_comparison", "cpu_baseline", "screen_precision"):
        assert callable(getattr(bench, name, None)), name
