"""FP64 CPU oracle for exact and c-approximate reverse k-ranks queries.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2504_13446_gb300``) and never imports it.

Arithmetic (the paper fixes no precision; these are the readings both sides use):

* Canonical score: s(u, x) = left-to-right FP64 sum of (double)u_k * (double)x_k
  (``rkr_oracle.c``).  Ranks compare canonical scores with strict ">" (Def. 1).
* Exact query (Def. 2): the k users with the smallest (rank, user index).
* Pre-processing (Alg. 1): items sorted by (descending norm, index); omega
  buckets of m // omega items, the first m % omega get one more; per-bucket
  sample positions are an input; thresholds t_j = f_min + (j-1) * ((f_max -
  f_min) / (tau - 1)); the table is kept as integer numerators N with
  T-hat = 1 + N / s.
* Query (Section 4.3): j = max{j : t_j <= u.q} (0 if none); r_up = T-hat_j
  (m + 1 when j = 0), r_low = T-hat_{j+1} (1 when j = tau); R_low_k and R_up_k
  are k-th smallest values.  Case A when c * R_low_k >= R_up_k: the k users with
  smallest (r_up, r_low, index).  Case B: U_c = {r_up <= c * R_low_k}, prune
  r_low > R_up_k, interpolate the rest linearly in u.q and take the
  k - |U_c| smallest (estimate, index).

Parity pins for every function here live in ``tests/test_oracle_*.py``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rkr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_library(force: bool = False) -> str:
    """Compile ``rkr_oracle.c`` with gcc (no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build_library())
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.rkro_dot.restype = ctypes.c_double
        lib.rkro_dot.argtypes = [P, P, i32]
        lib.rkro_norms.argtypes = [P, i64, i32, P]
        lib.rkro_scores.argtypes = [P, i64, P, i64, i32, i32, P]
        lib.rkro_ranks_literal.argtypes = [P, i64, P, i64, P, i64, i32, P]
        lib.rkro_ranks.argtypes = [P, i64, P, i64, P, i64, i32, i32, P]
        lib.rkro_fbounds_exact.argtypes = [P, i64, P, i64, i32, i32, P, P]
        lib.rkro_thresholds.argtypes = [ctypes.c_double, ctypes.c_double, i32, P]
        lib.rkro_rank_table.argtypes = [P, i64, i32, P, P, P, i32, P, P, i32, i32, P]
        _lib = lib
        return lib


def _nthreads() -> int:
    return max(1, os.cpu_count() or 1)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ scores

def dot(u, x) -> float:
    """Canonical score s(u, x) of two float32 vectors."""
    u, x = _f32(u), _f32(x)
    return _load().rkro_dot(_ptr(u), _ptr(x), u.shape[0])


def scores(U, X, nthreads: int | None = None) -> np.ndarray:
    """Matrix of canonical scores s(U_i, X_j), float64, shape (n, nx)."""
    U, X = _f32(U), _f32(X)
    out = np.empty((U.shape[0], X.shape[0]), dtype=np.float64)
    _load().rkro_scores(_ptr(U), U.shape[0], _ptr(X), X.shape[0], U.shape[1],
                        nthreads or _nthreads(), _ptr(out))
    return out


def norms(X) -> np.ndarray:
    """FP64 Euclidean norms sqrt(s(x, x)) of the rows of X (Alg. 1, first step)."""
    X = _f32(X)
    out = np.empty(X.shape[0], dtype=np.float64)
    _load().rkro_norms(_ptr(X), X.shape[0], X.shape[1], _ptr(out))
    return out


# ------------------------------------------------------------- exact path

def ranks_literal(U, P, Q) -> np.ndarray:
    """Def. 1 as a literal triple loop; int32 (n, nq).  Tiny inputs only."""
    U, P, Q = _f32(U), _f32(P), _f32(Q)
    out = np.empty((U.shape[0], Q.shape[0]), dtype=np.int32)
    _load().rkro_ranks_literal(_ptr(U), U.shape[0], _ptr(P), P.shape[0], _ptr(Q), Q.shape[0],
                               U.shape[1], _ptr(out))
    return out


def ranks(U, P, Q, nthreads: int | None = None) -> np.ndarray:
    """r(q, u, P) for every user and query (Def. 1); int32 (n, nq)."""
    U, P, Q = _f32(U), _f32(P), _f32(Q)
    out = np.empty((U.shape[0], Q.shape[0]), dtype=np.int32)
    _load().rkro_ranks(_ptr(U), U.shape[0], _ptr(P), P.shape[0], _ptr(Q), Q.shape[0],
                       U.shape[1], nthreads or _nthreads(), _ptr(out))
    return out


def select_exact(rank_col: np.ndarray, k: int, users: np.ndarray | None = None):
    """Def. 2 with the tie reading: the k users with smallest (rank, index).

    ``rank_col`` holds the ranks of ``users`` (default: all users 0..n-1).
    Returns (user ids, ranks), both int32, in (rank, index) order.
    """
    if users is None:
        users = np.arange(rank_col.shape[0], dtype=np.int64)
    order = np.lexsort((users, rank_col))[:k]
    return users[order].astype(np.int32), rank_col[order].astype(np.int32)


def exact_query(U, P, Q, k, subsets=None, nthreads: int | None = None):
    """Exact reverse k-ranks for every query: list of (users, ranks)."""
    R = ranks(U, P, Q, nthreads)
    k = np.broadcast_to(np.asarray(k), (Q.shape[0],))
    out = []
    for q in range(Q.shape[0]):
        if subsets is None:
            out.append(select_exact(R[:, q], int(k[q])))
        else:
            sub = np.asarray(subsets[q], dtype=np.int64)
            out.append(select_exact(R[sub, q], int(k[q]), sub))
    return out


# ------------------------------------------------- pre-processing (Alg. 1)

def bucket_sizes(m: int, omega: int) -> np.ndarray:
    """Alg. 1 "equally-sized" buckets: m // omega items, the first m % omega get one more."""
    base, extra = divmod(m, omega)
    return np.array([base + (1 if l < extra else 0) for l in range(omega)], dtype=np.int64)


def thresholds(fmin: float, fmax: float, tau: int) -> np.ndarray:
    """t_{u,1..tau} for one user (Section 4.2, step 2)."""
    t = np.empty(tau, dtype=np.float64)
    _load().rkro_thresholds(ctypes.c_double(fmin), ctypes.c_double(fmax), tau, _ptr(t))
    return t


def thresholds_all(fmin: np.ndarray, fmax: np.ndarray, tau: int) -> np.ndarray:
    """Thresholds of every user, float64 (n, tau), same operation order as ``thresholds``."""
    delta = (fmax - fmin) / float(tau - 1)
    step = np.arange(tau, dtype=np.float64)[None, :] * delta[:, None]
    return fmin[:, None] + step


def build_index(U, P, tau: int, omega: int, s: int, sample_pos: np.ndarray,
                fbounds: str = "exact", nthreads: int | None = None) -> dict:
    """Alg. 1: norms, sort, buckets, samples, thresholds, rank-table numerators.

    ``sample_pos`` is (omega, s) int32: positions inside each bucket (-1 = unused),
    as drawn by ``synth.sample_positions``.
    """
    U, P = _f32(U), _f32(P)
    n, d = U.shape
    m = P.shape[0]
    if tau < 2 or omega < 1 or s < 1 or omega > m:
        raise ValueError("need tau >= 2, 1 <= omega <= m, s >= 1")
    pn = norms(P)
    perm = np.lexsort((np.arange(m), -pn)).astype(np.int64)   # (descending norm, index)
    sizes = bucket_sizes(m, omega)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    samp_items, samp_count, weight = [], [], []
    for l in range(omega):
        pos = np.asarray(sample_pos[l])
        pos = pos[pos >= 0]
        take_all = sizes[l] <= s
        if take_all:
            if len(pos) != sizes[l]:
                raise ValueError("a bucket with at most s items must be taken whole")
        elif len(pos) != s or len(np.unique(pos)) != s or pos.max() >= sizes[l]:
            raise ValueError("need s distinct in-range positions per large bucket")
        samp_items.append(perm[offs[l] + pos])
        samp_count.append(len(pos))
        weight.append(s if take_all else int(sizes[l]))
    samp_items = np.concatenate(samp_items).astype(np.int64)
    samp_count = np.array(samp_count, dtype=np.int32)
    weight = np.array(weight, dtype=np.int64)
    if fbounds == "exact":
        fmin = np.empty(n, dtype=np.float64)
        fmax = np.empty(n, dtype=np.float64)
        _load().rkro_fbounds_exact(_ptr(U), n, _ptr(P), m, d, nthreads or _nthreads(),
                                   _ptr(fmin), _ptr(fmax))
    elif fbounds == "cs":
        # Footnote of Section 4.2: replace the scans by bounds of the domain;
        # here the Cauchy-Schwarz bound +-||u|| * max ||p|| of each user.
        fmax = norms(U) * pn[perm[0]]
        fmin = -fmax
    else:
        raise ValueError("fbounds must be 'exact' or 'cs'")
    S = np.ascontiguousarray(P[samp_items])
    N = np.empty((n, tau), dtype=np.uint32)
    _load().rkro_rank_table(_ptr(U), n, d, _ptr(S), _ptr(samp_count), _ptr(weight), omega,
                            _ptr(fmin), _ptr(fmax), tau, nthreads or _nthreads(), _ptr(N))
    return dict(n=n, m=m, d=d, tau=tau, omega=omega, s=s, perm=perm, pnorm=pn,
                sizes=sizes, offs=offs, samp_items=samp_items, samp_count=samp_count,
                weight=weight, fmin=fmin, fmax=fmax, N=N)


# ------------------------------------------------ query processing (4.3)

def lookup(index: dict, theta: np.ndarray, users: np.ndarray | None = None):
    """Step 1 bounds for one query: (j, N_low, N_up) per user.

    j = max{j : t_j <= theta} in 1..tau, or 0 when theta < t_1.
    r_up = 1 + N_up / s with N_up = N_j (m * s when j = 0);
    r_low = 1 + N_low / s with N_low = N_{j+1} (0 when j = tau).
    """
    tau, s, m = index["tau"], index["s"], index["m"]
    if users is None:
        users = np.arange(index["n"])
    fmin, fmax, N = index["fmin"][users], index["fmax"][users], index["N"][users]
    j = np.empty(len(users), dtype=np.int64)
    chunk = 1 << 14
    for lo in range(0, len(users), chunk):
        hi = min(len(users), lo + chunk)
        t = thresholds_all(fmin[lo:hi], fmax[lo:hi], tau)
        j[lo:hi] = np.sum(t <= theta[lo:hi, None], axis=1)
    rows = np.arange(len(users))
    n_up = np.where(j >= 1, N[rows, np.maximum(j - 1, 0)].astype(np.int64), m * s)
    n_low = np.where(j < tau, N[rows, np.minimum(j, tau - 1)].astype(np.int64), 0)
    return j, n_low, n_up


def interpolate(index: dict, theta, j, n_low, n_up, users):
    """Step 3 estimate: linear in u.q between (t_j, r_up) and (t_{j+1}, r_low).

    r_hat = r_up - (r_up - r_low) * (theta - t_j) / (t_{j+1} - t_j) for
    1 <= j <= tau - 1, else r_hat = r_up.  Every operation rounds to double.
    """
    tau, s = index["tau"], index["s"]
    fmin, fmax = index["fmin"][users], index["fmax"][users]
    delta = (fmax - fmin) / float(tau - 1)
    r_up = 1.0 + n_up.astype(np.float64) / float(s)
    r_low = 1.0 + n_low.astype(np.float64) / float(s)
    inside = (j >= 1) & (j <= tau - 1)
    jj = np.where(inside, j, 1).astype(np.float64)
    t_j = fmin + (jj - 1.0) * delta
    t_j1 = fmin + jj * delta
    with np.errstate(divide="ignore", invalid="ignore"):
        frac = (theta - t_j) / (t_j1 - t_j)
        est = r_up - (r_up - r_low) * frac
    return np.where(inside, est, r_up)


def approx_query_one(index: dict, theta: np.ndarray, k: int, c: float, users=None) -> dict:
    """Section 4.3 steps 1-3 for one query given canonical theta = s(u, q) per user."""
    s = index["s"]
    if users is None:
        users = np.arange(index["n"], dtype=np.int64)
    users = np.asarray(users, dtype=np.int64)
    j, n_low, n_up = lookup(index, theta, users)
    # Step 1: k-th smallest lower and upper bound.
    R_low = int(np.partition(n_low, k - 1)[k - 1])
    R_up = int(np.partition(n_up, k - 1)[k - 1])
    lhs = c * float(s + R_low)          # c * R_low_k, scaled by s
    est_all = None
    # Step 2: filtering.
    if lhs >= float(s + R_up):
        order = np.lexsort((users, n_low, n_up))[:k]
        case, chosen = 1, order
        nc = k
    else:
        in_c = (s + n_up).astype(np.float64) <= lhs
        idx_c = np.nonzero(in_c)[0]
        idx_c = idx_c[np.lexsort((users[idx_c], n_low[idx_c], n_up[idx_c]))]
        temp = np.nonzero((n_low <= R_up) & ~in_c)[0]
        # Step 3: interpolate the survivors and take the smallest estimates.
        est_t = interpolate(index, theta[temp], j[temp], n_low[temp], n_up[temp], users[temp])
        pick = temp[np.lexsort((users[temp], est_t))[: k - len(idx_c)]]
        case, chosen = 2, np.concatenate([idx_c, pick])
        nc = len(idx_c)
    est_all = interpolate(index, theta[chosen], j[chosen], n_low[chosen], n_up[chosen],
                          users[chosen])
    return dict(users=users[chosen].astype(np.int32), n_low=n_low[chosen].astype(np.uint32),
                n_up=n_up[chosen].astype(np.uint32), est=est_all, case=case, nc=nc,
                R_low=R_low, R_up=R_up)


def approx_query(index: dict, U, Q, k, c: float, subsets=None, nthreads=None):
    """c-approximate reverse k-ranks (Section 4.3) for every query of Q."""
    th = scores(U, Q, nthreads)
    k = np.broadcast_to(np.asarray(k), (Q.shape[0],))
    out = []
    for q in range(Q.shape[0]):
        if subsets is None:
            out.append(approx_query_one(index, th[:, q], int(k[q]), c))
        else:
            sub = np.asarray(subsets[q], dtype=np.int64)
            out.append(approx_query_one(index, th[sub, q], int(k[q]), c, sub))
    return out


# ----------------------------------------------------------------- metrics

def quality(exact_ranks_col: np.ndarray, returned: np.ndarray, k: int, c: float,
            users: np.ndarray | None = None) -> dict:
    """Accuracy and overall ratio (Section 5, "Criteria"), recall and c-bound violations.

    Positions pair the i-th smallest exact rank of the returned set with the
    i-th smallest exact rank overall (Def. 3).  Recall counts returned users
    whose exact rank is at most the k-th smallest exact rank.
    """
    if users is None:
        pool = exact_ranks_col
    else:
        pool = exact_ranks_col[np.asarray(users)]
    best = np.sort(pool, kind="stable")[:k].astype(np.float64)
    got = np.sort(exact_ranks_col[np.asarray(returned)], kind="stable").astype(np.float64)
    kth = best[-1]
    return dict(accuracy=float(np.mean(got <= c * best)),
                overall_ratio=float(np.mean(got / best)),
                recall=float(np.mean(got <= kth)),
                violations=int(np.sum(got > c * kth)))
