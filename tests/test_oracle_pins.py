"""Pins for the FP64 oracle: exact path (Def. 1, Def. 2) and canonical score.

Every check compares the oracle with something other than itself: exact
integer arithmetic in Python, a hand-derived rounding example, the
floating-point error bound of a left-to-right sum, or an invariant that
Def. 1 fixes (bounds, monotonicity, permutation and power-of-two scaling).
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _rows(rng, n, d, sigma=0.5):
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return (g * np.exp(sigma * rng.standard_normal((n, 1)))).astype(np.float32)


def _int_rows(rng, n, d, lo=-3, hi=4):
    return rng.integers(lo, hi, size=(n, d)).astype(np.float32)


def _py_rank(u, P, q):
    """Def. 1 with exact integer arithmetic (inputs hold small integers)."""
    iu = [int(v) for v in u]
    theta = sum(a * int(b) for a, b in zip(iu, q))
    return 1 + sum(1 for p in P if sum(a * int(b) for a, b in zip(iu, p)) > theta)


# ------------------------------------------------------------ canonical score

def test_canonical_left_to_right_golden():
    g = _golden("canonical_order.json")
    u = np.array(g["u"], dtype=np.float32)
    x = np.array(g["x"], dtype=np.float32)
    assert float(u[0]) == 2.0 ** 53
    assert oracle.dot(u, x) == g["canonical"]
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, x))
    assert exact == g["exact"]


def test_dot_integer_inputs_are_exact():
    rng = np.random.default_rng(1)
    for d in (1, 7, 32, 200):
        U = _int_rows(rng, 5, d, -1000, 1001)
        X = _int_rows(rng, 7, d, -1000, 1001)
        S = oracle.scores(U, X)
        for i in range(5):
            for j in range(7):
                want = sum(int(a) * int(b) for a, b in zip(U[i], X[j]))
                assert S[i, j] == want


def test_dot_within_left_to_right_error_bound():
    """|s - exact| <= gamma_{d-1} * sum |u_k x_k| (standard bound for recursive summation)."""
    rng = np.random.default_rng(2)
    for d in (3, 50, 200):
        U = _rows(rng, 4, d)
        X = _rows(rng, 4, d)
        S = oracle.scores(U, X)
        eps = 2.0 ** -53
        gamma = (d - 1) * eps / (1 - (d - 1) * eps)
        for i in range(4):
            for j in range(4):
                prods = [Fraction(float(a)) * Fraction(float(b)) for a, b in zip(U[i], X[j])]
                exact = sum(prods)
                bound = gamma * float(sum(abs(p) for p in prods))
                assert abs(Fraction(S[i, j]) - exact) <= Fraction(bound)


def test_scores_match_single_dot():
    rng = np.random.default_rng(3)
    U, X = _rows(rng, 6, 19), _rows(rng, 5, 19)
    S = oracle.scores(U, X, nthreads=3)
    for i in range(6):
        for j in range(5):
            assert S[i, j] == oracle.dot(U[i], X[j])


def test_norms_closed_form():
    X = np.array([[3, 4, 0], [0, 0, 0], [1, 2, 2], [2 ** -3, 0, 0]], dtype=np.float32)
    assert oracle.norms(X).tolist() == [5.0, 0.0, 3.0, 0.125]


# ----------------------------------------------------------------- ranks

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ranks_match_exact_integer_definition_with_ties(seed):
    rng = np.random.default_rng(seed)
    n, m, nq, d = 6, 25, 5, 4
    U = _int_rows(rng, n, d)
    P = _int_rows(rng, m, d)
    Q = np.vstack([P[:2], _int_rows(rng, nq - 2, d)])  # two queries inside P
    want = np.array([[_py_rank(U[i], P, Q[q]) for q in range(nq)] for i in range(n)])
    assert (oracle.ranks_literal(U, P, Q) == want).all()
    assert (oracle.ranks(U, P, Q, nthreads=2) == want).all()
    # integer data produces exact ties; make sure the case is exercised
    S = oracle.scores(U, P)
    th = oracle.scores(U, Q)
    assert any((S[i] == th[i, q]).sum() > 1 for i in range(n) for q in range(nq))


def test_sorted_ranks_equal_literal_definition_on_floats():
    rng = np.random.default_rng(4)
    U, P = _rows(rng, 9, 11), _rows(rng, 60, 11)
    Q = np.vstack([P[[3, 17]], _rows(rng, 4, 11)])
    assert (oracle.ranks(U, P, Q, nthreads=4) == oracle.ranks_literal(U, P, Q)).all()


def test_rank_bounds_and_queries_inside_P():
    rng = np.random.default_rng(5)
    m = 80
    U, P = _rows(rng, 30, 8), _rows(rng, m, 8)
    Q = np.vstack([P[:10], _rows(rng, 10, 8) * 3])
    R = oracle.ranks(U, P, Q)
    assert R.min() >= 1 and R.max() <= m + 1
    assert R[:, :10].max() <= m        # q in P never counts itself


def test_zero_user_has_rank_one_and_argmax_query_has_rank_one():
    rng = np.random.default_rng(6)
    P = _rows(rng, 50, 6)
    U = np.vstack([np.zeros((1, 6), np.float32), _rows(rng, 5, 6)])
    S = oracle.scores(U, P)
    best = P[np.argmax(S, axis=1)]
    R = oracle.ranks(U, P, np.vstack([best, _rows(rng, 3, 6)]))
    assert (R[0] == 1).all()
    assert all(R[i, i] == 1 for i in range(6))


def test_single_item():
    rng = np.random.default_rng(7)
    P = _rows(rng, 1, 5)
    U = _rows(rng, 8, 5)
    Q = np.vstack([P, -P, 2 * P])
    R = oracle.ranks(U, P, Q)
    S = oracle.scores(U, P)[:, 0]
    assert (R[:, 0] == 1).all()
    assert (R[:, 1] == np.where(S > -S, 2, 1)).all()
    assert (R[:, 2] == np.where(S > 2 * S, 2, 1)).all()


def test_permutation_invariance():
    rng = np.random.default_rng(8)
    U, P, Q = _rows(rng, 12, 9), _rows(rng, 70, 9), _rows(rng, 6, 9)
    R = oracle.ranks(U, P, Q)
    pp, pu = rng.permutation(70), rng.permutation(12)
    assert (oracle.ranks(U, P[pp], Q) == R).all()
    assert (oracle.ranks(U[pu], P, Q) == R[pu]).all()


def test_power_of_two_scaling_invariance():
    rng = np.random.default_rng(9)
    U, P, Q = _rows(rng, 12, 9), _rows(rng, 70, 9), _rows(rng, 6, 9)
    R = oracle.ranks(U, P, Q)
    assert (oracle.ranks(U * np.float32(8), P, Q) == R).all()
    assert (oracle.ranks(U, P * np.float32(0.25), Q * np.float32(0.25)) == R).all()


def test_rank_non_increasing_in_theta():
    rng = np.random.default_rng(10)
    U, P, Q = _rows(rng, 10, 7), _rows(rng, 90, 7), _rows(rng, 40, 7)
    R = oracle.ranks(U, P, Q)
    th = oracle.scores(U, Q)
    for i in range(10):
        order = np.argsort(th[i], kind="stable")
        assert (np.diff(R[i, order]) <= 0).all()


def test_exact_query_is_def2_with_index_tie_break():
    rng = np.random.default_rng(11)
    n, m, d = 40, 30, 3
    U, P = _int_rows(rng, n, d, -2, 3), _int_rows(rng, m, d, -2, 3)
    Q = P[:4]
    R = oracle.ranks(U, P, Q)
    for q, (users, rk) in enumerate(oracle.exact_query(U, P, Q, 7)):
        assert len(users) == 7 and len(set(users.tolist())) == 7
        assert (R[users, q] == rk).all()
        others = np.setdiff1d(np.arange(n), users)
        assert rk.max() <= R[others, q].min()                  # Def. 2
        key = [(int(r), int(u)) for r, u in zip(rk, users)]
        assert key == sorted(key)
        tied = [u for u in others if R[u, q] == rk.max()]
        assert all(u > users[rk == rk.max()].max() for u in tied)  # index tie-break
