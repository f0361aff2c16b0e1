"""Pins of the FP64 network reference: explicit loops, central finite
differences, a hand-computed Adam step, and a planted mistake that the
finite-difference pin must catch."""
import numpy as np

from oracle import mlp


def _tiny(seed=0):
    rng = np.random.default_rng(seed)
    params = mlp.glorot_uniform(rng, [5, 4, 3, 2])
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    X = rng.standard_normal((6, 5))
    T = rng.standard_normal((6, 2))
    return params, X, T


def test_forward_matches_explicit_loops():
    params, X, T = _tiny(1)
    Y, _ = mlp.forward(params, X)
    for s in range(X.shape[0]):
        h = list(X[s])
        for l, (W, b) in enumerate(params):
            z = [sum(W[o, i] * h[i] for i in range(len(h))) + b[o] for o in range(W.shape[0])]
            h = [max(v, 0.0) for v in z] if l + 1 < len(params) else z
        assert np.allclose(Y[s], h, rtol=1e-13, atol=1e-13)
    assert abs(mlp.loss(params, X, T) - np.mean((Y - T) ** 2)) < 1e-15


def _fd(params, X, T, l, which, idx, h=1e-6):
    def with_delta(d):
        ps = [(W.copy(), b.copy()) for W, b in params]
        arr = ps[l][which]
        arr[idx] += d
        return mlp.loss(ps, X, T)
    return (with_delta(h) - with_delta(-h)) / (2 * h)


def test_gradients_match_central_differences():
    params, X, T = _tiny(2)
    _, grads = mlp.gradients(params, X, T)
    rng = np.random.default_rng(0)
    for l in range(len(params)):
        for which in (0, 1):
            shape = params[l][which].shape
            for _ in range(6):
                idx = tuple(int(rng.integers(0, s)) for s in shape)
                g = grads[l][which][idx]
                assert abs(g - _fd(params, X, T, l, which, idx)) <= 1e-7 * (1 + abs(g))


def test_finite_difference_pin_detects_a_planted_mistake(monkeypatch):
    params, X, T = _tiny(3)
    real = mlp.gradients

    def wrong(p, x, t):  # drops the ReLU mask (a plausible backprop mistake)
        Y, inputs = mlp.forward(p, x)
        B, out = Y.shape
        G = 2.0 * (Y - t) / (B * out)
        grads = [None] * len(p)
        for l in range(len(p) - 1, -1, -1):
            grads[l] = (G.T @ inputs[l], G.sum(axis=0))
            if l > 0:
                G = G @ p[l][0]
        return 0.0, grads

    monkeypatch.setattr(mlp, "gradients", wrong)
    _, grads = mlp.gradients(params, X, T)
    monkeypatch.setattr(mlp, "gradients", real)
    worst = 0.0
    for l in range(len(params)):
        for idx in np.ndindex(params[l][0].shape):
            worst = max(worst, abs(grads[l][0][idx] - _fd(params, X, T, l, 0, idx)))
    assert worst > 1e-4


def test_adam_first_step_by_hand():
    W = np.array([[1.0, -2.0]])
    b = np.array([0.5])
    g = [(np.array([[0.3, -0.1]]), np.array([2.0]))]
    opt = mlp.Adam([(W, b)], lr=0.01, beta1=0.9, beta2=0.999, eps=1e-8)
    (W1, b1), = opt.step([(W, b)], g)
    # first step: m_hat = g, v_hat = g^2, so the step is lr * g / (|g| + eps)
    assert np.allclose(W1, W - 0.01 * np.sign(g[0][0]) * np.abs(g[0][0]) / (np.abs(g[0][0]) + 1e-8))
    assert np.allclose(b1, b - 0.01 * 2.0 / (2.0 + 1e-8))
    # second step with the same gradient keeps the same direction and size
    (W2, _), = opt.step([(W1, b1)], g)
    assert np.allclose(W2 - W1, W1 - W, rtol=1e-6)
