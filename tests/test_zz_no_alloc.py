"""rkr_screen_scores_static (the allocation-free screen) against rkr_screen_scores.

Collected last on purpose: it must also pass after every other GPU test has run
in the same process.  Both entries run the same staging, tile-bound and screen
kernels, so their outputs agree bit for bit; the static one is called twice in
a row to show that its shared scratch carries nothing from one call to the next.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")
torch = pytest.importorskip("torch")


def _rows(rng, n, d):
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return (g * np.exp(0.7 * rng.standard_normal((n, 1)))).astype(np.float32)


@pytest.mark.parametrize("split", [False, True])
def test_static_screen_matches_allocating_screen(split):
    rng = np.random.default_rng(11)
    cases = [(300, 517, 100), (129, 260, 37)]   # two calls in a row, different shapes
    for n, mx, d in cases:
        U, X = _rows(rng, n, d), _rows(rng, mx, d)
        s_ref, b_ref = rkr.rkr_screen_scores(U, X, split=split)
        Ud, Xd = torch.from_numpy(U).cuda(), torch.from_numpy(X).cuda()
        for _ in range(2):
            s = torch.full((n, mx), float("nan"), device="cuda")
            b = torch.full((n, mx), float("nan"), device="cuda")
            allocs = rkr.device_allocations()
            rkr.rkr_screen_scores_static(Ud, Xd, s, b, split=split)
            # the library requested no device memory for the call
            assert rkr.device_allocations() == allocs
            assert (s.cpu().numpy() == s_ref).all()
            assert (b.cpu().numpy() == b_ref).all()


def test_allocation_counter_moves_for_the_allocating_screen():
    rng = np.random.default_rng(3)
    U, X = _rows(rng, 40, 16), _rows(rng, 50, 16)
    allocs = rkr.device_allocations()
    rkr.rkr_screen_scores(U, X)
    assert rkr.device_allocations() > allocs


def test_static_screen_rejects_a_width_mismatch():
    U = torch.zeros((4, 8), device="cuda")
    X = torch.zeros((4, 6), device="cuda")
    out = torch.empty((4, 4), device="cuda")
    with pytest.raises(rkr.RKRError) as e:
        rkr.rkr_screen_scores_static(U, X, out, out.clone())
    assert e.value.status == 1 and "columns" in str(e.value)


def test_static_screen_rejects_sizes_beyond_its_scratch():
    d = 256
    n = mx = 9000   # about 19 MB of scratch against the 16 MiB array
    U = torch.zeros((n, d), device="cuda")
    X = torch.zeros((mx, 1), device="cuda").expand(mx, d).contiguous()
    s = torch.empty((1, 1), device="cuda")
    with pytest.raises(rkr.RKRError) as e:
        lib = rkr.load()
        rkr._check(lib.rkr_screen_scores_static(U.data_ptr(), n, X.data_ptr(), mx, d, 1,
                                                s.data_ptr(), s.data_ptr(), None))
    assert e.value.status == 1 and "static limit" in str(e.value)


def test_static_screen_rejects_host_pointers():
    U = np.zeros((4, 8), dtype=np.float32)
    out = np.zeros((4, 4), dtype=np.float32)
    lib = rkr.load()
    with pytest.raises(rkr.RKRError) as e:
        rkr._check(lib.rkr_screen_scores_static(U.ctypes.data, 4, U.ctypes.data, 4, 8, 0,
                                                out.ctypes.data, out.ctypes.data, None))
    assert e.value.status == 1


def test_static_screen_rejects_the_fp8_form():
    U = torch.zeros((4, 8), device="cuda")
    out = torch.empty((4, 4), device="cuda")
    lib = rkr.load()
    with pytest.raises(rkr.RKRError) as e:
        rkr._check(lib.rkr_screen_scores_static(U.data_ptr(), 4, U.data_ptr(), 4, 8, 2,
                                                out.data_ptr(), out.data_ptr(), None))
    assert e.value.status == 1
