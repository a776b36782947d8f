"""The premise of the exact path's early termination over the norm-sorted items,
checked on the CPU with the oracle's canonical scores.

Alg. 1 sorts P by descending norm.  For a user u and a query q, the number of
items of the first m1 of that order scoring above u.q is at most the number of
all items above it (a count over a subset of P).  Given any k users whose full
counts are known, the k-th smallest of those counts caps the k-th smallest
count of all users, so a user whose prefix count already exceeds the cap
cannot be among the k smallest (count, user) pairs: dropping every such user
leaves Def. 2's answer unchanged.  The GPU pass takes the cap from the users
with the smallest possible prefix counts; here the cap comes from the users
with the smallest prefix counts, and from a random k of them, and both must
give the oracle's answer.
"""

import numpy as np

import oracle


def _rows(rng, n, d, lean):
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    x = g * np.exp(0.5 * rng.standard_normal((n, 1)))
    x[:, 0] += lean
    return x.astype(np.float32)


def test_prefix_counts_drop_only_users_outside_the_answer():
    rng = np.random.default_rng(17)
    dropped = checked = 0
    for trial in range(6):
        n, m, d = 300, int(rng.integers(200, 500)), 12
        U, P = _rows(rng, n, d, 0.0), _rows(rng, m, d, 0.6 * (trial % 2))
        Q = np.vstack([1e-3 * P[:3], np.zeros((1, d), np.float32), P[3:5]])
        S = oracle.scores(U, P)                       # n x m canonical scores
        theta = oracle.scores(U, Q)                   # n x nq
        order = np.lexsort((np.arange(m), -oracle.norms(P)))
        above = S[:, order][:, None, :] > theta[:, :, None]   # n x nq x m, norm order
        full = above.sum(axis=2)
        R = oracle.ranks(U, P, Q)
        assert (R == full + 1).all()
        for q in range(Q.shape[0]):
            k = int(rng.integers(1, 30))
            want_u, want_r = oracle.select_exact(R[:, q], k)
            for frac in (0.125, 0.25, 0.5):
                m1 = max(1, int(m * frac))
                pre = above[:, q, :m1].sum(axis=1)
                assert (pre <= full[:, q]).all()
                for pick in ("smallest", "random"):
                    if pick == "smallest":
                        chosen = np.argsort(pre, kind="stable")[:max(k, 8)]
                    else:
                        chosen = rng.choice(n, size=k, replace=False)
                    cap = np.sort(full[chosen, q])[k - 1]
                    keep = np.nonzero(pre <= cap)[0]
                    got_u, got_r = oracle.select_exact(R[keep, q], k, keep)
                    assert (got_u == want_u).all() and (got_r == want_r).all()
                    dropped += n - len(keep)
                    checked += n
    assert dropped > checked // 10   # the bound does drop users (most on leaning items)
