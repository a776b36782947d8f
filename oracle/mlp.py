"""FP64 reference of the monotone rank regressor used as a learned pruner.

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` and ``__graft_entry__.smoke()`` may
import this module.  It shares no code with the CUDA path.

The regressor predicts y = log r(q, u, P) from features of a (user, query) pair:
``x`` (the non-monotone features: a fixed random projection of the user's unit
direction and the log of the user's norm) and ``t`` (the user-normalised score
u.q / ||u||).  A larger score cannot mean a larger rank (Def. 1), so the output
is made non-increasing in t by construction:

    h1 = relu(W1 x - softplus(A) t + b1)          (the t weights are <= 0)
    h2 = relu(softplus(V2) h1 + b2)               (later weights are >= 0)
    y  = softplus(v3) . h2 + b3

Every path from t to y then has a non-positive weight product through
non-decreasing activations.  Loss: mean squared error 0.5 * mean((y - target)^2).

Parameters are a dict of float64 arrays:
    W1 (H, F), A (H,), b1 (H,), V2 (H, H), b2 (H,), v3 (H,), b3 ().
"""

from __future__ import annotations

import numpy as np

ORDER = ("W1", "A", "b1", "V2", "b2", "v3", "b3")


def softplus(z):
    z = np.asarray(z, dtype=np.float64)
    return np.where(z > 30.0, z, np.log1p(np.exp(np.minimum(z, 30.0))))


def sigmoid(z):
    z = np.asarray(z, dtype=np.float64)
    return 1.0 / (1.0 + np.exp(-z))


def shapes(F: int, H: int) -> dict:
    return dict(W1=(H, F), A=(H,), b1=(H,), V2=(H, H), b2=(H,), v3=(H,), b3=())


def flatten(params: dict) -> np.ndarray:
    """Parameters in the fixed order W1, A, b1, V2, b2, v3, b3 (row-major)."""
    return np.concatenate([np.asarray(params[k], np.float64).ravel() for k in ORDER])


def unflatten(vec, F: int, H: int) -> dict:
    out, o = {}, 0
    for k in ORDER:
        shp = shapes(F, H)[k]
        size = int(np.prod(shp)) if shp else 1
        out[k] = np.asarray(vec[o:o + size], np.float64).reshape(shp)
        o += size
    return out


def forward(p: dict, X, t):
    """Predicted log ranks and the activations needed by backward."""
    X = np.asarray(X, np.float64)
    t = np.asarray(t, np.float64).reshape(-1)
    wt = -softplus(p["A"])
    z1 = X @ p["W1"].T + np.outer(t, wt) + p["b1"]
    h1 = np.maximum(z1, 0.0)
    W2 = softplus(p["V2"])
    z2 = h1 @ W2.T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    w3 = softplus(p["v3"])
    y = h2 @ w3 + p["b3"]
    return y, dict(X=X, t=t, z1=z1, h1=h1, z2=z2, h2=h2, W2=W2, w3=w3)


def loss_and_grads(p: dict, X, t, target):
    """0.5 * mean((y - target)^2) and its gradient with respect to every parameter."""
    y, c = forward(p, X, t)
    target = np.asarray(target, np.float64).reshape(-1)
    B = y.shape[0]
    r = y - target
    loss = 0.5 * float(np.mean(r * r))
    dy = r / B
    g = {}
    g["b3"] = np.array(dy.sum())
    dw3 = c["h2"].T @ dy
    g["v3"] = dw3 * sigmoid(p["v3"])
    dz2 = np.outer(dy, c["w3"]) * (c["z2"] > 0)
    g["b2"] = dz2.sum(axis=0)
    dW2 = dz2.T @ c["h1"]
    g["V2"] = dW2 * sigmoid(p["V2"])
    dz1 = (dz2 @ c["W2"]) * (c["z1"] > 0)
    g["b1"] = dz1.sum(axis=0)
    g["W1"] = dz1.T @ c["X"]
    dwt = dz1.T @ c["t"]
    g["A"] = dwt * (-sigmoid(p["A"]))
    return loss, g


def init_params(F: int, H: int, seed: int) -> dict:
    """A reproducible starting point (Gaussian weights scaled by fan-in)."""
    rng = np.random.default_rng(seed)
    return dict(W1=rng.standard_normal((H, F)) / np.sqrt(F),
                A=np.full(H, -1.0) + 0.1 * rng.standard_normal(H),
                b1=np.zeros(H),
                V2=np.log(np.expm1(np.full((H, H), 1.0 / H))) + 0.1 * rng.standard_normal((H, H)),
                b2=np.zeros(H),
                v3=np.log(np.expm1(np.full(H, 1.0 / np.sqrt(H)))),
                b3=np.array(0.0))
