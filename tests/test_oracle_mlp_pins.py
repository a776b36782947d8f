"""Pins of the FP64 reference of the learned pruner's regressor (oracle/mlp.py).

The analytic gradient is checked against central finite differences (an
independent computation), monotonicity in the score input against a grid, and
the forward pass against a hand-computed one-unit network.
"""

import numpy as np
import pytest

from oracle import mlp


def _small(F=5, H=7, seed=0):
    p = mlp.init_params(F, H, seed)
    rng = np.random.default_rng(seed + 1)
    # move away from the symmetric start so every path is exercised
    for k in p:
        p[k] = p[k] + 0.3 * rng.standard_normal(np.shape(p[k]))
    X = rng.standard_normal((9, F))
    t = rng.standard_normal(9)
    y = rng.standard_normal(9)
    return p, X, t, y


def test_gradient_matches_central_differences():
    p, X, t, y = _small()
    loss, g = mlp.loss_and_grads(p, X, t, y)
    h = 1e-6
    for k in mlp.ORDER:
        flat = np.asarray(p[k], np.float64).ravel()
        gk = np.asarray(g[k]).ravel()
        for i in range(flat.size):
            q = {kk: np.array(v, copy=True) for kk, v in p.items()}
            qf = q[k].ravel() if q[k].shape else q[k].reshape(1)
            qf[i] += h
            q[k] = qf.reshape(np.shape(p[k]))
            lp, _ = mlp.loss_and_grads(q, X, t, y)
            qf[i] -= 2 * h
            q[k] = qf.reshape(np.shape(p[k]))
            lm, _ = mlp.loss_and_grads(q, X, t, y)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gk[i]) <= 1e-6 + 1e-5 * abs(fd), (k, i, fd, gk[i])


def test_output_non_increasing_in_score():
    p, X, _, _ = _small(seed=3)
    grid = np.linspace(-4, 4, 401)
    for row in X:
        y, _ = mlp.forward(p, np.repeat(row[None, :], grid.size, axis=0), grid)
        assert (np.diff(y) <= 1e-12).all()


def test_one_unit_network_by_hand():
    p = dict(W1=np.array([[2.0, -1.0]]), A=np.array([0.0]), b1=np.array([0.5]),
             V2=np.array([[0.0]]), b2=np.array([0.25]), v3=np.array([0.0]), b3=np.array(1.0))
    sp0 = np.log(2.0)   # softplus(0)
    X = np.array([[1.0, 1.0], [0.0, 3.0]])
    t = np.array([0.5, 1.0])
    y, _ = mlp.forward(p, X, t)
    # unit 1: z1 = 2 - 1 - ln2 * 0.5 + 0.5; z2 = ln2 * relu(z1) + 0.25; y = ln2 * relu(z2) + 1
    z1 = np.array([2 - 1 - sp0 * 0.5 + 0.5, -3 - sp0 * 1.0 + 0.5])
    z2 = sp0 * np.maximum(z1, 0) + 0.25
    want = sp0 * np.maximum(z2, 0) + 1.0
    assert np.allclose(y, want, rtol=0, atol=1e-15)


def test_flatten_round_trip():
    p = mlp.init_params(4, 3, 2)
    q = mlp.unflatten(mlp.flatten(p), 4, 3)
    for k in mlp.ORDER:
        assert np.array_equal(np.asarray(p[k]), np.asarray(q[k]))
