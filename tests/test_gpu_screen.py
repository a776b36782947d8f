"""The tcgen05 BF16 screen: every screened score lies within its bound of the
canonical FP64 score, in single (hi.hi) and split (hi.hi + hi.lo + lo.hi) form."""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")


def _rows(rng, n, d, sigma=0.7):
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return (g * np.exp(sigma * rng.standard_normal((n, 1)))).astype(np.float32)


@pytest.mark.parametrize("n,mx,d", [(300, 700, 32), (129, 257, 100), (260, 513, 200),
                                    (77, 300, 37), (128, 256, 256)])
@pytest.mark.parametrize("split", [False, True])
def test_screen_within_bound(n, mx, d, split):
    rng = np.random.default_rng(n + mx + d)
    U, X = _rows(rng, n, d), _rows(rng, mx, d)
    s, b = rkr.rkr_screen_scores(U, X, split=split)
    S = oracle.scores(U, X)
    err = np.abs(s.astype(np.float64) - S)
    assert np.isfinite(s).all() and (b > 0).all()
    ratio = err / b
    assert ratio.max() <= 1.0, f"max error/bound {ratio.max()}"
    # the bound uses the largest item norm of each 256-column tile
    xn = np.linalg.norm(X, axis=1)
    tile_max = np.repeat([xn[i:i + 256].max() for i in range(0, mx, 256)], 256)[:mx]
    scale = np.linalg.norm(U, axis=1)[:, None] * tile_max[None, :]
    rel = (b / scale).max()
    assert rel < (2e-2 if not split else 1e-4), rel
    # the screen is not trivially loose: typical error far below the bound
    assert np.median(ratio) < 0.5


@pytest.mark.parametrize("split", [False, True])
def test_screen_within_bound_on_the_bench_items(split):
    """The bound at the bench workload's width and length: 64 users of its
    generator (Gaussian mixture, d = 200) against all 100,000 of its items,
    every one of the 6.4M pairs within its bound of the canonical score."""
    import synth
    w = synth.make_workload("approx", n=64, nq=1)
    s, b = rkr.rkr_screen_scores(w.U, w.P, split=split)
    S = oracle.scores(w.U, w.P)
    ratio = np.abs(s.astype(np.float64) - S) / b
    assert np.isfinite(s).all() and (b > 0).all()
    assert ratio.max() <= 1.0, f"max error/bound {ratio.max()}"
    assert np.median(ratio) < 0.5


@pytest.mark.parametrize("d", [200, 32, 72])
def test_split_over_concatenated_operands_is_bit_identical(d):
    """The split product run as one pass over [hi | lo | hi] x [lo | hi | hi] (K = 3 K')
    issues the same MMAs in the same order as the three K' segments: equal bits."""
    rng = np.random.default_rng(d)
    U, X = _rows(rng, 300, d), _rows(rng, 700, d)
    before = rkr.rkr_tuning_get()
    try:
        rkr.rkr_tuning_set(split_cat=1)
        s1, b1 = rkr.rkr_screen_scores(U, X, split=True)
        rkr.rkr_tuning_set(split_cat=0)
        s0, b0 = rkr.rkr_screen_scores(U, X, split=True)
    finally:
        rkr.rkr_tuning_set(**before)
    assert (s1 == s0).all() and (b1 == b0).all()


def test_screen_integer_data_is_exact_when_representable():
    """Small integers are exact in bf16 and their products sum exactly in FP32."""
    rng = np.random.default_rng(1)
    U = rng.integers(-8, 9, size=(140, 48)).astype(np.float32)
    X = rng.integers(-8, 9, size=(300, 48)).astype(np.float32)
    s, b = rkr.rkr_screen_scores(U, X)
    assert (s.astype(np.float64) == oracle.scores(U, X)).all()


@pytest.mark.parametrize("n,mx,d", [(300, 700, 32), (129, 257, 100), (128, 512, 128),
                                    (77, 300, 37), (260, 513, 200)])
def test_fp8_screen_within_bound(n, mx, d):
    """E4M3 operands with per-row power-of-two scales (one product, kind::f8f6f4): every
    scaled score lies within its bound of the canonical score; the bound is of the order
    of the E4M3 unit roundoff (2^-4) times the norms, far looser than the BF16 forms."""
    rng = np.random.default_rng(n * 7 + mx + d)
    U, X = _rows(rng, n, d), _rows(rng, mx, d)
    s, b = rkr.rkr_screen_scores(U, X, split=2)
    S = oracle.scores(U, X)
    err = np.abs(s.astype(np.float64) - S)
    assert np.isfinite(s).all() and (b > 0).all()
    ratio = err / b
    assert ratio.max() <= 1.0, f"max error/bound {ratio.max()}"
    xn = np.linalg.norm(X, axis=1)
    tile_max = np.repeat([xn[i:i + 256].max() for i in range(0, mx, 256)], 256)[:mx]
    rel = (b / (np.linalg.norm(U, axis=1)[:, None] * tile_max[None, :])).max()
    assert rel < 0.5, rel
    # the FP8 product tracks the score: typical error well below the bound
    assert np.median(ratio) < 0.5
    # ... and is much coarser than the split BF16 product
    s3, b3 = rkr.rkr_screen_scores(U, X, split=True)
    assert np.median(b) > 10 * np.median(b3)
