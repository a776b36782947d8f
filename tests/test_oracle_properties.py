"""Property tests of the oracle's ranks (Def. 1) on inputs drawn by hypothesis.

Small float matrices (entries on a coarse binary grid, so that some products tie
exactly) check, for every draw: the sorted-score ranks equal the literal count
of Def. 1; 1 <= r <= m + 1, and r <= m for a query that is an item of P (its own
copy never counts); invariance under permutations of U and of P; invariance
under scaling U, and P with Q, by powers of two (exact in FP64); and, for a fixed
user, ranks that never increase as u.q grows.
"""

import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import given, settings  # noqa: E402


def _matrix(draw, rows, d):
    # multiples of 1/8 in [-4, 4]: products and sums stay exact in FP64, and ties occur
    vals = draw(st.lists(st.integers(-32, 32), min_size=rows * d, max_size=rows * d))
    return (np.array(vals, dtype=np.float64).reshape(rows, d) / 8.0).astype(np.float32)


@st.composite
def problems(draw):
    n = draw(st.integers(1, 8))
    m = draw(st.integers(1, 12))
    d = draw(st.integers(1, 5))
    U, P = _matrix(draw, n, d), _matrix(draw, m, d)
    fresh = _matrix(draw, draw(st.integers(0, 3)), d)
    pick = draw(st.lists(st.integers(0, m - 1), min_size=1, max_size=3))
    Q = np.vstack([P[pick], fresh]).astype(np.float32)
    seed = draw(st.integers(0, 2 ** 31 - 1))
    return U, P, Q, len(pick), seed


@settings(max_examples=80, deadline=None)
@given(problems())
def test_rank_properties(prob):
    U, P, Q, nfrom_p, seed = prob
    rng = np.random.default_rng(seed)
    m = P.shape[0]
    R = oracle.ranks(U, P, Q)
    assert (R == oracle.ranks_literal(U, P, Q)).all()
    assert R.min() >= 1 and R.max() <= m + 1
    assert (R[:, :nfrom_p] <= m).all()
    # permutations of U and of P
    pu, pp = rng.permutation(U.shape[0]), rng.permutation(m)
    assert (oracle.ranks(U[pu], P[pp], Q) == R[pu]).all()
    # powers of two: u.p and u.q scale alike and exactly
    a, b = 2.0 ** int(rng.integers(-3, 4)), 2.0 ** int(rng.integers(-3, 4))
    Us = (U * a).astype(np.float32)
    Ps, Qs = (P * b).astype(np.float32), (Q * b).astype(np.float32)
    assert (oracle.ranks(Us, Ps, Qs) == R).all()
    # for a fixed user, a larger u.q never has a larger rank
    S = oracle.scores(U, Q)
    for i in range(U.shape[0]):
        order = np.argsort(S[i], kind="stable")
        assert (np.diff(R[i, order].astype(np.int64)) <= 0).all()
