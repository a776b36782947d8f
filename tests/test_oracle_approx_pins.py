"""Pins for the oracle's transcription of Alg. 1 and Section 4.3.

Checks against: the exact rank-table definition (Section 4.2, step 3) with
exact integer arithmetic when every item is sampled; the sandwich inequality of
Section 4.1; unbiasedness of Eq. 1 over many sample draws; the Fig. 1 lookup;
hand-built tables whose Case A / Case B outcome is worked out by hand; and the
structural facts of Lemma 1 and the filtering step.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(rng, n, d, sigma=0.5):
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return (g * np.exp(sigma * rng.standard_normal((n, 1)))).astype(np.float32)


def _take_all_positions(m, omega, s):
    sizes = oracle.bucket_sizes(m, omega)
    assert sizes.max() <= s
    return synth.sample_positions(0, sizes, s)


def _index_from_table(fmin, fmax, N, tau, s, m):
    n = len(fmin)
    return dict(n=n, m=m, tau=tau, s=s, fmin=np.asarray(fmin, float), fmax=np.asarray(fmax, float),
                N=np.asarray(N, dtype=np.uint32))


# --------------------------------------------------------------- pre-processing

def test_bucket_sizes_equal_with_remainder_first():
    assert oracle.bucket_sizes(10, 3).tolist() == [4, 3, 3]
    assert oracle.bucket_sizes(9, 3).tolist() == [3, 3, 3]
    assert oracle.bucket_sizes(5, 5).tolist() == [1] * 5


def test_thresholds_closed_form():
    t = oracle.thresholds(0.0, 9.0, 10)
    assert t.tolist() == [float(j) for j in range(10)]
    t = oracle.thresholds(-1.0, 1.0, 5)
    assert t.tolist() == [-1.0, -0.5, 0.0, 0.5, 1.0]
    t = oracle.thresholds(2.5, 2.5, 4)       # f_max = f_min: every threshold is f_min
    assert t.tolist() == [2.5] * 4
    fmin = np.array([0.0, -1.0, 0.3]); fmax = np.array([9.0, 1.0, 0.7])
    for i, tau in enumerate((10, 5, 7)):
        assert (oracle.thresholds_all(fmin[i:i + 1], fmax[i:i + 1], tau)[0]
                == oracle.thresholds(fmin[i], fmax[i], tau)).all()


def test_sort_is_descending_norm_then_index():
    P = np.array([[1, 0], [0, 2], [2, 0], [0, 1], [3, 4]], dtype=np.float32)
    idx = oracle.build_index(P[:1], P, tau=2, omega=1, s=5,
                             sample_pos=_take_all_positions(5, 1, 5))
    assert idx["perm"].tolist() == [4, 1, 2, 0, 3]


@pytest.mark.parametrize("fb", ["exact", "cs"])
def test_table_equals_exact_counts_when_every_item_is_sampled(fb):
    """s >= |P_l| for all l: Eq. 1 collapses to the exact T of Section 4.2, step 3."""
    rng = np.random.default_rng(3)
    n, m, d, tau, omega, s = 7, 41, 3, 9, 4, 11
    U = rng.integers(-3, 4, size=(n, d)).astype(np.float32)
    P = rng.integers(-3, 4, size=(m, d)).astype(np.float32)
    idx = oracle.build_index(U, P, tau, omega, s, _take_all_positions(m, omega, s), fbounds=fb)
    for i in range(n):
        iu = [int(v) for v in U[i]]
        sc = [sum(a * int(b) for a, b in zip(iu, p)) for p in P]
        if fb == "exact":
            assert idx["fmax"][i] == max(sc) and idx["fmin"][i] == min(sc)
        t = oracle.thresholds(idx["fmin"][i], idx["fmax"][i], tau)
        for j in range(tau):
            count = sum(1 for v in sc if v > t[j])      # exact int-vs-double comparison
            assert idx["N"][i, j] == s * count


def test_table_structure_with_sampling():
    rng = np.random.default_rng(4)
    n, m, d, tau, omega, s = 20, 500, 6, 30, 5, 17
    U, P = _rows(rng, n, d), _rows(rng, m, d)
    pos = synth.sample_positions(9, oracle.bucket_sizes(m, omega), s)
    idx = oracle.build_index(U, P, tau, omega, s, pos)
    N = idx["N"].astype(np.int64)
    assert (np.diff(N, axis=1) <= 0).all()            # T-hat non-increasing in j
    assert N.max() <= m * s                            # T-hat <= m + 1
    assert (N % np.gcd.reduce(idx["weight"]) == 0).all()
    # the sampled items are the right ones: inside their bucket of the sorted order
    offs, perm = idx["offs"], idx["perm"]
    items = idx["samp_items"].reshape(omega, s)
    for l in range(omega):
        assert set(items[l]) <= set(perm[offs[l]:offs[l + 1]].tolist())


def test_estimator_is_unbiased():
    """E[T-hat] = T (end of Section 4.2): average over many independent sample draws."""
    rng = np.random.default_rng(5)
    n, m, d, tau, omega, s = 4, 240, 5, 12, 4, 15
    U, P = _rows(rng, n, d), _rows(rng, m, d)
    full = oracle.build_index(U, P, tau, 1, m, _take_all_positions(m, 1, m))
    exact = full["N"].astype(np.float64) / m           # exact counts #{p : s > t_j}
    sizes = oracle.bucket_sizes(m, omega)
    draws = 400
    acc = np.zeros((n, tau))
    sq = np.zeros((n, tau))
    for seed in range(draws):
        pos = synth.sample_positions(1000 + seed, sizes, s)
        est = oracle.build_index(U, P, tau, omega, s, pos)["N"].astype(np.float64) / s
        acc += est
        sq += est ** 2
    mean = acc / draws
    sd = np.sqrt(np.maximum(sq / draws - mean ** 2, 1e-12) / draws)
    assert np.all(np.abs(mean - exact) <= 5 * sd + 1e-9)


# ------------------------------------------------------------------- queries

def test_fig1_lookup_bounds():
    g = json.load(open(os.path.join(GOLDEN, "fig1_lookup.json")))
    N = np.array([g["T_row"]], dtype=np.int64) - 1
    idx = _index_from_table([g["fmin"]], [g["fmax"]], N * g["s"], g["tau"], g["s"], m=100)
    j, n_low, n_up = oracle.lookup(idx, np.array([g["theta"]]))
    assert j[0] == g["expect_j"]
    assert 1 + n_low[0] / g["s"] == g["expect_r_low"]
    assert 1 + n_up[0] / g["s"] == g["expect_r_up"]


def test_lookup_edges_and_equality():
    idx = _index_from_table([0.0], [4.0], [[8, 6, 3, 1, 0]], tau=5, s=2, m=9)
    j, lo, up = oracle.lookup(idx, np.array([-0.5]))
    assert (j[0], lo[0], up[0]) == (0, 8, 9 * 2)        # below t_1: r_up = m + 1
    j, lo, up = oracle.lookup(idx, np.array([4.0]))
    assert (j[0], lo[0], up[0]) == (5, 0, 0)            # at t_tau: r_low = 1
    j, lo, up = oracle.lookup(idx, np.array([2.0]))
    assert (j[0], lo[0], up[0]) == (3, 1, 3)            # equality takes the larger j


def test_interpolation_closed_form():
    idx = _index_from_table([0.0], [4.0], [[8, 6, 3, 1, 0]], tau=5, s=2, m=9)
    th = np.array([2.5])
    j, lo, up = oracle.lookup(idx, th)
    est = oracle.interpolate(idx, th, j, lo, up, np.array([0]))
    # r_up = 1 + 3/2 = 2.5, r_low = 1 + 1/2 = 1.5, halfway -> 2.0
    assert est[0] == 2.0
    est = oracle.interpolate(idx, np.array([9.0]), np.array([5]), np.array([0]), np.array([0]),
                             np.array([0]))
    assert est[0] == 1.0                                  # outside the grid: r_up


def _hand_index():
    # five users, one query direction; thresholds 0..4 for everyone (tau = 5, s = 1)
    N = [[40, 30, 20, 10, 0],
         [40, 30, 20, 10, 0],
         [40, 35, 33, 31, 30],
         [45, 44, 43, 42, 41],
         [40, 12, 11, 10, 9]]
    return _index_from_table([0.0] * 5, [4.0] * 5, N, tau=5, s=1, m=50)


def test_case_a_by_hand():
    idx = _hand_index()
    theta = np.array([3.5, 2.5, 3.5, 3.5, 0.5])
    # j = 4,3,4,4,1 -> (r_low, r_up) = (1,11), (11,21), (31,32), (42,43), (13,41)
    out = oracle.approx_query_one(idx, theta, k=2, c=2.0)
    # numerators: R_low_2 = 10 (rank 11), R_up_2 = 20 (rank 21); 2 * 11 = 22 >= 21: Case A
    assert out["case"] == 1 and out["R_low"] == 10 and out["R_up"] == 20
    assert out["users"].tolist() == [0, 1]


def test_case_b_by_hand():
    idx = _hand_index()
    theta = np.array([3.5, 1.5, 0.5, 3.5, 2.5])
    # j = 4,2,1,4,3 -> (r_low, r_up) = (1,11), (21,31), (36,41), (42,43), (11,12)
    out = oracle.approx_query_one(idx, theta, k=3, c=1.2)
    # R_low_3 = 21 (N 20), R_up_3 = 31 (N 30); 1.2 * 21 = 25.2 < 31: Case B
    assert out["case"] == 2 and out["R_low"] == 20 and out["R_up"] == 30
    # U_c = {r_up <= 25.2} = {0, 4} in (r_up, r_low, index) order; users 2 and 3
    # are pruned (r_low > 31); user 1 is the only survivor and fills the last slot
    assert out["nc"] == 2 and out["users"].tolist() == [0, 4, 1]
    assert out["est"][2] == 31 - 10 * 0.5
    out = oracle.approx_query_one(idx, theta, k=4, c=1.5)
    # R_low_4 = 37 (N 36), R_up_4 = 43 (N 42): 1.5 * 37 = 55.5 >= 43: Case A
    assert out["case"] == 1 and out["users"].tolist() == [0, 4, 1, 2]


def test_case_b_step3_by_hand():
    N = [[10, 8, 6, 4, 2],
         [10, 9, 8, 7, 6],
         [10, 9, 8, 7, 6],
         [10, 5, 4, 3, 2]]
    idx = _index_from_table([0.0] * 4, [4.0] * 4, N, tau=5, s=1, m=20)
    theta = np.array([3.5, 2.25, 2.75, 0.5])
    # j = 4,3,3,1; (N_low, N_up) = (2,4), (7,8), (7,8), (5,10)
    out = oracle.approx_query_one(idx, theta, k=2, c=1.0)
    # R_low_2 = 5, R_up_2 = 8; 1 * 6 < 9: Case B.  U_c = {N_up <= 5} = {0}.
    # prune N_low > 8: none; U_temp = {1, 2, 3}; estimates 1 + 8 - 1*0.25 = 8.75,
    # 9 - 0.75 = 8.25, 11 - 5*0.5 = 8.5 -> user 2 (8.25) completes the answer
    assert out["case"] == 2 and out["nc"] == 1
    assert out["users"].tolist() == [0, 2]
    assert out["est"].tolist() == [1 + 4 - 2 * 0.5, 8.25]


def test_guarantees_with_exact_table():
    """With every item sampled the table is exact, r_low <= r <= r_up holds, and
    the filter of Lemma 1 keeps the c-bound for every user returned at step 2."""
    rng = np.random.default_rng(12)
    n, m, d, tau = 300, 120, 6, 40
    U, P = _rows(rng, n, d), _rows(rng, m, d)
    Q = np.vstack([P[:10], _rows(rng, 10, d)])
    idx = oracle.build_index(U, P, tau, 3, 40, _take_all_positions(m, 3, 40))
    R = oracle.ranks(U, P, Q)
    th = oracle.scores(U, Q)
    c = 1.5
    for q in range(Q.shape[0]):
        j, n_low, n_up = oracle.lookup(idx, th[:, q])
        r_low = 1 + n_low / idx["s"]
        r_up = 1 + n_up / idx["s"]
        assert (r_low <= R[:, q]).all() and (R[:, q] <= r_up).all()
        for k in (1, 5, 20):
            out = oracle.approx_query_one(idx, th[:, q], k, c)
            users = out["users"]
            assert len(users) == k and len(set(users.tolist())) == k
            kth = np.sort(R[:, q])[k - 1]
            step2 = users[:out["nc"]]
            assert (R[step2, q] <= c * kth).all()
            if out["case"] == 2:
                assert out["nc"] < k


def test_quality_metrics_identity():
    R = np.array([5, 3, 9, 3, 1, 7])
    q = oracle.quality(R, np.array([4, 1, 3]), 3, 2.0)
    assert q == dict(accuracy=1.0, overall_ratio=1.0, recall=1.0, violations=0)
    q = oracle.quality(R, np.array([4, 1, 2]), 3, 2.0)
    assert q["recall"] == 2 / 3 and q["violations"] == 1
    assert q["overall_ratio"] == (1 + 1 + 3) / 3
