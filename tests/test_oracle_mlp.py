"""Pins for the oracle's rank-predictor network: hand-written gradients against
central finite differences, the asymmetric loss, and that Adam reduces the
loss on a learnable target."""
import numpy as np

from oracle import mlp as M


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    F, B = 7, 11
    params = M.init_params(F, seed=1)
    X = rng.standard_normal((B, F))
    t = rng.standard_normal(B) * 2.0
    alpha = 4.0
    y, cache = M.forward(params, X)
    grads = M.backward(params, cache, y, t, alpha)
    h = 1e-6
    for li in range(len(params)):
        for pi in range(2):
            P = params[li][pi]
            flat = P.reshape(-1)
            picks = rng.choice(flat.size, size=min(6, flat.size), replace=False)
            for idx in picks:
                old = flat[idx]
                flat[idx] = old + h
                lp = M.loss(M.forward(params, X)[0], t, alpha)
                flat[idx] = old - h
                lm = M.loss(M.forward(params, X)[0], t, alpha)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[li][pi].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (li, pi, idx, fd, an)


def test_asymmetric_loss_penalises_under_prediction():
    t = np.array([3.0, 3.0])
    assert M.loss(np.array([2.0, 2.0]), t, 4.0) == 4.0
    assert M.loss(np.array([4.0, 4.0]), t, 4.0) == 1.0


def test_adam_learns_linear_target():
    rng = np.random.default_rng(2)
    F = 5
    X = rng.standard_normal((256, F))
    t = X @ np.array([1.0, -2.0, 0.5, 0.0, 3.0]) + 4.0
    params = M.init_params(F, seed=3)
    state = {}
    l0 = M.loss(M.forward(params, X)[0], t, 2.0)
    for _ in range(300):
        y, c = M.forward(params, X)
        g = M.backward(params, c, y, t, 2.0)
        M.adam_step(params, g, state, lr=3e-3)
    l1 = M.loss(M.forward(params, X)[0], t, 2.0)
    assert l1 < 0.05 * l0
