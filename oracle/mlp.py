"""Per-bond rank predictor: a multilayer perceptron with three hidden layers of
width 64 and ReLU, hand-written forward and backward passes in FP64, and an
Adam update.  Not in the paper (the nearest
relative is the coarse-grained rank of Sec. 5.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Model:   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3),
         y  = W4 h3 + b4        (y = predicted log2 of the bond rank)
Loss:    L = (1/B) sum_b w_b (y_b - t_b)^2 with w_b = alpha where the model
         under-predicts (y_b < t_b) and 1 elsewhere.
Weights: W_l of shape (out, in) row-major; a batch is X of shape (B, F).
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64
DEPTH = 3


def init_params(n_features: int, seed: int = 0):
    """He-normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    sizes = [n_features] + [HIDDEN] * DEPTH + [1]
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = rng.standard_normal((b, a)) * np.sqrt(2.0 / a)
        params.append([W, np.zeros(b)])
    return params


def forward(params, X):
    """Returns (y, cache) with y of shape (B,)."""
    acts = [X]
    pre = []
    h = X
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        pre.append(z)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
        acts.append(h)
    return h[:, 0], (acts, pre)


def loss(y, t, alpha: float):
    w = np.where(y < t, alpha, 1.0)
    return float(np.mean(w * (y - t) ** 2))


def backward(params, cache, y, t, alpha: float):
    """Gradients of `loss` with respect to every W_l and b_l."""
    acts, pre = cache
    B = y.shape[0]
    w = np.where(y < t, alpha, 1.0)
    g = (2.0 / B) * w * (y - t)
    g = g[:, None]
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        if li < len(params) - 1:
            g = g * (pre[li] > 0.0)
        gW = g.T @ acts[li]
        gb = g.sum(axis=0)
        grads[li] = [gW, gb]
        g = g @ W
    return grads


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), in place.  `state` is a dict holding
    the step count and the first/second moment estimates."""
    if not state:
        state["t"] = 0
        state["m"] = [[np.zeros_like(p) for p in layer] for layer in params]
        state["v"] = [[np.zeros_like(p) for p in layer] for layer in params]
    state["t"] += 1
    t = state["t"]
    for li, layer in enumerate(params):
        for pi in range(2):
            g = grads[li][pi]
            m = state["m"][li][pi] = beta1 * state["m"][li][pi] + (1 - beta1) * g
            v = state["v"][li][pi] = beta2 * state["v"][li][pi] + (1 - beta2) * g * g
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            layer[pi] = layer[pi] - lr * mh / (np.sqrt(vh) + eps)
    return params
