"""The learned pruner's regressor on the GPU against the FP64 reference (oracle/mlp.py).

The kernels round operands to BF16 and accumulate in FP32, so outputs and
gradients are compared with a relative tolerance derived from the BF16 unit
roundoff (2^-8) over the layer depths; monotonicity in the score input is exact.
"""

import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

rkr = pytest.importorskip("paper_2504_13446_gb300")


def _setup(F=9, H=32, B=200, seed=1):
    p = mlp.init_params(F, H, seed)
    rng = np.random.default_rng(seed)
    for k in p:
        p[k] = p[k] + 0.2 * rng.standard_normal(np.shape(p[k]))
    flat = mlp.flatten(p).astype(np.float32)
    p32 = mlp.unflatten(flat.astype(np.float64), F, H)   # the exact parameters the GPU holds
    X = rng.standard_normal((B, F)).astype(np.float32)
    t = rng.standard_normal(B).astype(np.float32)
    y = rng.standard_normal(B).astype(np.float32) * 2
    return p32, flat, X, t, y


def test_forward_and_gradients_match_fp64_reference():
    F, H = 9, 32
    p, flat, X, t, target = _setup(F, H)
    net = rkr.Pruner(F, H, seed=0)
    net.set_params(flat)
    assert np.array_equal(net.get_params(), flat)
    y_gpu = net.forward(X, t)
    y_ref, _ = mlp.forward(p, X.astype(np.float64), t.astype(np.float64))
    assert np.abs(y_gpu - y_ref).max() <= 3e-2 * (1 + np.abs(y_ref).max())
    loss_gpu, g_gpu = net.loss_grads(X, t, target)
    loss_ref, g_ref = mlp.loss_and_grads(p, X.astype(np.float64), t.astype(np.float64), target)
    assert abs(loss_gpu - loss_ref) <= 3e-2 * (1 + loss_ref)
    gf = mlp.unflatten(g_gpu.astype(np.float64), F, H)
    for k in mlp.ORDER:
        a, b = np.asarray(gf[k]).ravel(), np.asarray(g_ref[k]).ravel()
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        assert rel < 5e-2, (k, rel)


def test_output_non_increasing_in_score_on_gpu():
    F, H = 9, 32
    _, flat, X, _, _ = _setup(F, H, B=8, seed=4)
    net = rkr.Pruner(F, H)
    net.set_params(flat)
    grid = np.linspace(-3, 3, 257).astype(np.float32)
    for row in X:
        y = net.forward(np.repeat(row[None, :], grid.size, axis=0), grid)
        assert (np.diff(y) <= 0).all()


def test_training_reduces_the_loss():
    rng = np.random.default_rng(7)
    F, H, n = 9, 64, 20000
    X = rng.standard_normal((n, F)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    # a monotone target: larger score, smaller log rank
    target = (3.0 - 1.5 * t + 0.3 * X[:, 0] + 0.1 * np.abs(X[:, 1])).astype(np.float32)
    net = rkr.Pruner(F, H, seed=3)
    before, _ = net.loss_grads(X[:4096], t[:4096], target[:4096])
    net.train(X, t, target, epochs=8, batch=1024, lr=3e-3, seed=1)
    after, _ = net.loss_grads(X[:4096], t[:4096], target[:4096])
    assert after < 0.3 * before and after < 0.15, (before, after)
