"""A bounded device wait that runs out (SURVEY-style fault test without a GPU fault).

rkr_set_wait_limit(0) makes the epilogue warps of the tensor-core screens give
up at their first accumulator wait.  The shape below has one row block and one
column tile, so the screen runs on the single-CTA kernel: its MMA warp still
consumes every TMA stage and its MMAs complete before the CTA exits, so nothing
is in flight when the kernel returns.  The call must report RKR_ETIMEOUT, and
with the default limit restored the next calls must succeed with unchanged
results.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")
torch = pytest.importorskip("torch")

ETIMEOUT = 4


def _rows(rng, n, d):
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return (g * np.exp(0.5 * rng.standard_normal((n, 1)))).astype(np.float32)


def test_wait_limit_gives_timeout_then_next_call_succeeds():
    rng = np.random.default_rng(5)
    U, X = _rows(rng, 100, 64), _rows(rng, 200, 64)
    s_ref, b_ref = rkr.rkr_screen_scores(U, X, split=True)
    try:
        rkr.rkr_set_wait_limit(0)
        with pytest.raises(rkr.RKRError) as e:
            rkr.rkr_screen_scores(U, X, split=True)
        assert e.value.status == ETIMEOUT
    finally:
        rkr.rkr_set_wait_limit(-1)
    torch.cuda.synchronize()   # the context is still usable
    s, b = rkr.rkr_screen_scores(U, X, split=True)
    assert (s == s_ref).all() and (b == b_ref).all()
    # and a whole query path still runs
    P = _rows(rng, 300, 64)
    with rkr.Index(U, P, tau=16, omega=3, s=20, exact_table=True) as idx:
        users, ranks, off, _ = idx.query_exact(P[:4], 5)
    assert len(users) == 20 and (ranks >= 1).all()


def test_wait_limit_argument_checks():
    with pytest.raises(rkr.RKRError):
        rkr.rkr_set_wait_limit(1 << 40)
    rkr.rkr_set_wait_limit(-5)   # any negative value restores the default
