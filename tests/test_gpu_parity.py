"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Exact path: users and ranks bit-identical (Def. 1, Def. 2 with index
tie-break).  Approximate path: norm order, f_min/f_max, the table numerators of
Alg. 1 and every output of the Section 4.3 query steps bit-identical to the
oracle's transcription, on the same seeded inputs and sample positions.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")


def _rows(rng, n, d, sigma=0.5):
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return (g * np.exp(sigma * rng.standard_normal((n, 1)))).astype(np.float32)


def build_pair(U, P, tau, omega, s, *, seed=0, fbounds="exact", floor_rank=0):
    pos = synth.sample_positions(seed, oracle.bucket_sizes(P.shape[0], omega), s)
    ora = oracle.build_index(U, P, tau, omega, s, pos, fbounds=fbounds)
    gpu = rkr.Index(U, P, tau=tau, omega=omega, s=s, fbounds=fbounds, sample_pos=pos,
                    exact_table=True, floor_rank=floor_rank)
    return ora, gpu


def check_index(ora, gpu):
    assert (gpu.export("perm") == ora["perm"]).all()
    assert (gpu.export("pnorm") == ora["pnorm"]).all()
    assert (gpu.export("samples") == ora["samp_items"]).all()
    assert (gpu.export("fmin") == ora["fmin"]).all()
    assert (gpu.export("fmax") == ora["fmax"]).all()
    N = gpu.export("table")
    bad = np.argwhere(N != ora["N"])
    assert len(bad) == 0, f"{len(bad)} table cells differ, first {bad[:5].tolist()}"


def check_exact_table(ora, gpu, U, P, floor_rank=0):
    """The exact count bounds: XLO <= #{p : s(u,p) > x_j} <= XHI on each user's tail grid, where
    x_0 is the sampled table's threshold at its last column whose estimated count
    reaches the floor rank and x_{G-1} = f_max (same threshold formula)."""
    m, s, tau = P.shape[0], ora["s"], ora["tau"]
    R = floor_rank or max(2048, m // 16)
    S = oracle.scores(U, P)
    grid = gpu.export("xgrid")
    xlo, xhi = gpu.export("xlo"), gpu.export("xhi")
    G = xlo.shape[1]
    for i in range(U.shape[0]):
        Nrow = ora["N"][i].astype(np.int64)
        below = np.nonzero(Nrow < s * R)[0]
        a = below[0] if len(below) else tau
        fl = a - 1 if a > 0 else 0
        g0 = oracle.thresholds(ora["fmin"][i], ora["fmax"][i], tau)[fl]
        x = oracle.thresholds(g0, ora["fmax"][i], G)
        assert grid[i, 0] == g0 and grid[i, 1] == (ora["fmax"][i] - g0) / float(G - 1), i
        srt = np.sort(S[i])
        cnt = S.shape[1] - np.searchsorted(srt, x, side="right")
        assert (xlo[i] <= cnt).all() and (cnt <= xhi[i]).all(), i
        tight = np.mean(xlo == xhi)
    assert tight > 0.5, tight   # most counts are decided by the screen alone


def check_exact(U, P, Q, k, gpu):
    users, ranks, off, stats = gpu.query_exact(Q, k)
    want = oracle.exact_query(U, P, Q, k)
    for q, (wu, wr) in enumerate(want):
        gu, gr = users[off[q]:off[q + 1]], ranks[off[q]:off[q + 1]]
        assert (gu == wu).all() and (gr == wr).all(), (q, gu[:8], wu[:8], gr[:8], wr[:8])
    return stats


def check_approx(U, Q, k, c, ora, gpu):
    out = gpu.query_approx(Q, k, c)
    want = oracle.approx_query(ora, U, Q, k, c)
    off = out["offsets"]
    for q, w in enumerate(want):
        sl = slice(off[q], off[q + 1])
        assert out["case"][q] == w["case"] and out["nc"][q] == w["nc"], q
        assert (out["users"][sl] == w["users"]).all(), (q, out["users"][sl][:8], w["users"][:8])
        assert (out["n_low"][sl] == w["n_low"]).all(), q
        assert (out["n_up"][sl] == w["n_up"]).all(), q
        assert (out["est"][sl] == w["est"]).all(), q
    return out


def test_exact_small_workload_full():
    """2,000 users x 5,000 items, d = 32, 16 queries from P, k = 10: the whole answer."""
    w = synth.make_workload("exact_small")
    ora, gpu = build_pair(w.U, w.P, 64, 8, 50)
    check_index(ora, gpu)
    check_exact_table(ora, gpu, w.U, w.P)
    check_exact(w.U, w.P, w.Q, w.k, gpu)
    check_approx(w.U, w.Q, w.k, 2.0, ora, gpu)


@pytest.mark.parametrize("n,m,d,nq", [(1037, 777, 37, 33), (3001, 1200, 100, 70)])
def test_ragged_sizes(n, m, d, nq):
    rng = np.random.default_rng(n)
    U, P = _rows(rng, n, d, 0.7), _rows(rng, m, d, 0.7)
    Q = np.vstack([P[rng.choice(m, nq // 2, replace=False)], _rows(rng, nq - nq // 2, d, 0.7)])
    k = rng.integers(1, 60, size=nq).astype(np.int32)
    ora, gpu = build_pair(U, P, 37, 7, 23, seed=3)
    check_index(ora, gpu)
    check_exact(U, P, Q, k, gpu)
    for c in (1.0, 1.5, 3.0):
        check_approx(U, Q, k, c, ora, gpu)


def test_approx_workload_shape_scaled():
    """The c-approximate workload's generator and parameters (tau 500, omega 10, s 100,
    d 200, mixture data, k in {10, 50, 100}) at reduced n, m."""
    w = synth.make_workload("approx", n=12000, m=3000, nq=24)
    ora, gpu = build_pair(w.U, w.P, w.tau, w.omega, w.s, seed=w.seed)
    check_index(ora, gpu)
    check_exact_table(ora, gpu, w.U, w.P)
    check_approx(w.U, w.Q, w.k, w.c, ora, gpu)
    check_exact(w.U, w.P, w.Q, w.k, gpu)


def test_integer_data_with_exact_ties():
    """Small-integer vectors make exact score ties everywhere: strict > of Def. 1."""
    rng = np.random.default_rng(9)
    U = rng.integers(-3, 4, size=(700, 6)).astype(np.float32)
    P = rng.integers(-3, 4, size=(400, 6)).astype(np.float32)
    Q = np.vstack([P[:10], rng.integers(-3, 4, size=(6, 6)).astype(np.float32)])
    k = np.array([1, 5, 50, 200] * 4, dtype=np.int32)
    ora, gpu = build_pair(U, P, 12, 4, 30)
    check_index(ora, gpu)
    check_exact(U, P, Q, k, gpu)
    check_approx(U, Q, k, 1.0, ora, gpu)
    check_approx(U, Q, k, 2.0, ora, gpu)


@pytest.mark.parametrize("fb", ["exact", "cs"])
def test_take_all_buckets_and_bounds_variants(fb):
    rng = np.random.default_rng(4)
    U, P = _rows(rng, 500, 16), _rows(rng, 90, 16)
    Q = _rows(rng, 9, 16)
    ora, gpu = build_pair(U, P, 20, 9, 10, fbounds=fb)   # every bucket taken whole
    check_index(ora, gpu)
    check_approx(U, Q, 7, 1.2, ora, gpu)
    check_exact(U, P, Q, 7, gpu)


def test_degenerate_sizes():
    rng = np.random.default_rng(5)
    # one user, one item, d = 1, k = n
    U, P = _rows(rng, 1, 1), _rows(rng, 1, 1)
    Q = np.vstack([P, -P, _rows(rng, 2, 1)])
    ora, gpu = build_pair(U, P, 2, 1, 1)
    check_index(ora, gpu)
    check_exact(U, P, Q, 1, gpu)
    check_approx(U, Q, 1, 1.0, ora, gpu)
    # k = n, omega = m (one item per bucket), tau = 2
    U, P = _rows(rng, 40, 3), _rows(rng, 25, 3)
    Q = _rows(rng, 5, 3)
    ora, gpu = build_pair(U, P, 2, 25, 1)
    check_index(ora, gpu)
    check_exact(U, P, Q, 40, gpu)
    check_approx(U, Q, 40, 1.0, ora, gpu)


def test_device_and_host_arrays_agree():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    U, P, Q = _rows(rng, 900, 24), _rows(rng, 500, 24), _rows(rng, 12, 24)
    gpu = rkr.Index(torch.from_numpy(U).cuda(), torch.from_numpy(P).cuda(), tau=30, omega=5,
                    s=20, exact_table=True)
    host = gpu.query_exact(Q, 9)
    dev = gpu.query_exact(torch.from_numpy(Q).cuda(), torch.full((12,), 9, dtype=torch.int32,
                                                                 device="cuda"), device=True)
    assert (dev[0].cpu().numpy() == host[0]).all() and (dev[1].cpu().numpy() == host[1]).all()
    a = gpu.query_approx(Q, 9, 1.5)
    b = gpu.query_approx(torch.from_numpy(Q).cuda(), 9, 1.5, device=True)
    assert (b["users"].cpu().numpy() == a["users"]).all()


def test_invalid_arguments_return_status():
    rng = np.random.default_rng(7)
    U, P, Q = _rows(rng, 50, 4), _rows(rng, 30, 4), _rows(rng, 3, 4)
    gpu = rkr.Index(U, P, tau=8, omega=3, s=5)
    for bad_k in (0, 51):
        with pytest.raises(rkr.RKRError) as e:
            gpu.query_exact(Q, bad_k)
        assert e.value.status == 1
    with pytest.raises(rkr.RKRError):
        gpu.query_approx(Q, 3, 0.5)
    Qn = Q.copy()
    Qn[1, 2] = np.nan
    with pytest.raises(rkr.RKRError):
        gpu.query_exact(Qn, 3)
    with pytest.raises(rkr.RKRError):
        rkr.Index(U, P, tau=1, omega=3, s=5)
    with pytest.raises(rkr.RKRError):
        rkr.Index(U, P, tau=8, omega=31, s=5)
    # the index stays usable after errors
    check_exact(U, P, Q, 4, gpu)


@pytest.mark.parametrize("level", ["0", "3", "40"])
def test_skip_level_leaves_results_unchanged(monkeypatch, level):
    """Pairs whose lower rank bound lies above the skip level are left out by one compare;
    queries whose cutoff lies above it are screened again in full.  Level 0 makes almost
    every query deep, 40 turns skipping off: the answers stay those of the oracle."""
    monkeypatch.setenv("RKR_SKIP_LEVEL", level)
    w = synth.make_workload("approx", n=12000, m=3000, nq=40)
    ora, gpu = build_pair(w.U, w.P, w.tau, w.omega, w.s, seed=w.seed)
    out = check_approx(w.U, w.Q, w.k, w.c, ora, gpu)
    st = check_exact(w.U, w.P, w.Q, w.k, gpu)
    if level == "40":
        assert out["stats"].deep_queries == 0 and st.deep_queries == 0
    if level == "0":
        assert out["stats"].deep_queries > 0 and st.deep_queries > 0


@pytest.mark.parametrize("floor_rank", [8, 40])
def test_recount_below_the_tail_lists(floor_rank):
    """A low floor rank leaves most candidates below their user's tail list, and
    tiny-norm queries put u.q near the middle of every user's scores, so the
    cutoff is wide open: ranks come from the count-interval recount and the
    resolution of its survivors."""
    rng = np.random.default_rng(floor_rank)
    U, P = _rows(rng, 3000, 48), _rows(rng, 4000, 48)
    Q = np.vstack([P[:6], 1e-3 * P[6:9], _rows(rng, 3, 48), np.zeros((1, 48), np.float32)])
    k = np.array([1, 5, 20, 60, 7, 13, 30, 2, 50, 9, 25, 3, 11], dtype=np.int32)
    ora, gpu = build_pair(U, P, 40, 6, 30, floor_rank=floor_rank)
    check_exact_table(ora, gpu, U, P, floor_rank=floor_rank)
    st = check_exact(U, P, Q, k, gpu)
    assert st.recounted > 0 and st.wide_queries > 0


def test_prefix_prune_over_norm_sorted_items():
    """Early termination over the norm-sorted items: tiny-norm and zero queries
    make every user a recount candidate, so those queries take the prefix pass
    (every candidate screened against the first m / p items, the most promising
    recounted over all of P for the cap, the others dropped when their prefix
    count already exceeds it).  The items lean towards one direction, so users'
    counts at u.q = 0 spread from a few hundred to most of P.  Answers equal the
    oracle's for every prefix length and with the pass switched off."""
    rng = np.random.default_rng(5)
    d = 48
    lean = np.zeros(d, np.float32)
    lean[0] = 0.5
    U, P = _rows(rng, 6000, d), (_rows(rng, 5000, d) + lean).astype(np.float32)
    Q = np.vstack([1e-3 * P[:4], np.zeros((1, d), np.float32), P[4:7], _rows(rng, 2, d)])
    k = np.array([1, 10, 32, 4, 17, 5, 40, 8, 3, 21], dtype=np.int32)
    before = rkr.rkr_tuning_get()
    try:
        ora, gpu = build_pair(U, P, 40, 6, 30, floor_rank=40)
        ref = gpu.query_exact(Q, k)
        for p in (0, 2, 4, 16):
            rkr.rkr_tuning_set(rc_prefix=p)
            st = check_exact(U, P, Q, k, gpu)
            got = gpu.query_exact(Q, k)
            assert (got[0] == ref[0]).all() and (got[1] == ref[1]).all(), p
            if p == 0:
                assert st.prefix_rows == 0 and st.prefix_pruned == 0
                continue
            assert st.prefix_rows >= 5 * 2048, p      # the five wide queries
            if p == 2:
                assert st.prefix_pruned > st.prefix_rows // 2, st.prefix_pruned
            if p == 4:
                assert st.prefix_pruned > 0
    finally:
        rkr.rkr_tuning_set(**before)


@pytest.mark.parametrize("split_first", [1, 0])
def test_recount_many_thresholds_per_user(split_first):
    """Forty tiny-norm queries make every user a candidate of each of them, so
    the recount (with multi-threshold segments switched on) compares each
    user's scores with forty sorted thresholds (two segments of 20).  Items of P among the queries (one of them
    twice) tie exactly with their own threshold and sit at a known position
    among the others; a copy of a tiny query gives equal thresholds."""
    rng = np.random.default_rng(77)
    U, P = _rows(rng, 1500, 40), _rows(rng, 3000, 40)
    scales = np.geomspace(1e-4, 3e-2, 38).astype(np.float32)
    tiny = scales[:, None] * P[100:138]
    Q = np.vstack([tiny, tiny[5:6], P[3:4], P[3:4], P[10:14], _rows(rng, 4, 40)])
    k = rng.integers(1, 80, size=Q.shape[0]).astype(np.int32)
    before = rkr.rkr_tuning_get()
    try:
        rkr.rkr_tuning_set(rc_single_first=split_first, rc_seg_min=4)
        ora, gpu = build_pair(U, P, 40, 6, 30, floor_rank=8)
        st = check_exact(U, P, Q, k, gpu)
        assert st.recounted > 0 and st.recount_users > 0
        assert st.recounted > 10 * st.recount_users   # many thresholds per user
    finally:
        rkr.rkr_tuning_set(**before)


def check_deep_grid(gpu, U, P):
    """The deep count grid: DLO <= #{p : s(u,p) > y_c} <= DHI for every user and
    grid point, y_c = y_0 + c * step from the exported grid."""
    S = oracle.scores(U, P)
    grid = gpu.export("dgrid")
    dlo, dhi = gpu.export("dlo"), gpu.export("dhi")
    G = dlo.shape[1]
    x0 = gpu.export("xgrid")[:, 0]
    assert G == rkr.DEEP_GRID
    for i in range(U.shape[0]):
        assert grid[i, 0] <= x0[i], i
        y = grid[i, 0] + np.arange(G, dtype=np.float64) * grid[i, 1]
        srt = np.sort(S[i])
        cnt = S.shape[1] - np.searchsorted(srt, y, side="right")
        assert (dlo[i] <= cnt).all() and (cnt <= dhi[i]).all(), i


@pytest.mark.parametrize("floor_rank", [8, 40])
def test_deep_grid_bounds_and_fewer_recounts(floor_rank):
    """exact_table = 2 adds the deep count grid below the tail lists: its bounds
    hold for every user against brute-force counts, the answers stay the
    oracle's, and queries deep below the floor rank recount fewer candidates."""
    rng = np.random.default_rng(100 + floor_rank)
    U, P = _rows(rng, 3000, 48), _rows(rng, 4000, 48)
    Q = np.vstack([P[:6], 1e-3 * P[6:9], _rows(rng, 3, 48), np.zeros((1, 48), np.float32)])
    k = np.array([1, 5, 20, 60, 7, 13, 30, 2, 50, 9, 25, 3, 11], dtype=np.int32)
    pos = synth.sample_positions(0, oracle.bucket_sizes(P.shape[0], 6), 30)
    plain = rkr.Index(U, P, tau=40, omega=6, s=30, sample_pos=pos, exact_table=True,
                      floor_rank=floor_rank)
    deep = rkr.Index(U, P, tau=40, omega=6, s=30, sample_pos=pos, exact_table=2,
                     floor_rank=floor_rank)
    check_deep_grid(deep, U, P)
    st_plain = check_exact(U, P, Q, k, plain)
    st_deep = check_exact(U, P, Q, k, deep)
    assert st_deep.recounted < st_plain.recounted, (st_deep.recounted, st_plain.recounted)
    with pytest.raises(rkr.RKRError):
        rkr.Index(U, P, tau=40, omega=6, s=30, sample_pos=pos, exact_table=3)
