"""Pins of the learned-guess network oracle: finite differences, Adam's closed
first step, and the linear regime.  CPU only."""

import numpy as np

from oracle import mlp_oracle as M


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    params = M.init_params(5, 7, hidden=6, seed=1)
    params = [(W + 0.05 * rng.standard_normal(W.shape), b + 0.1 * rng.standard_normal(b.shape))
              for W, b in params]
    X = rng.standard_normal((4, 5))
    T = rng.standard_normal((4, 7))
    grads = M.backward(params, X, T)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            flat = arr.reshape(-1)
            gflat = g.reshape(-1)
            for idx in range(0, flat.size, max(1, flat.size // 9)):
                old = flat[idx]
                flat[idx] = old + h
                lp = M.loss(params, X, T)
                flat[idx] = old - h
                lm = M.loss(params, X, T)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - gflat[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_closed_form():
    params = M.init_params(3, 2, hidden=4, seed=2)
    grads = [(np.full_like(W, 0.3), np.full_like(b, -2.0)) for W, b in params]
    before = [(W.copy(), b.copy()) for W, b in params]
    M.adam_step(params, grads, {}, lr=0.01, eps=1e-8)
    for (W0, b0), (W1, b1) in zip(before, params):
        assert np.allclose(W1 - W0, -0.01 * 0.3 / (0.3 + 1e-8), rtol=1e-12)
        assert np.allclose(b1 - b0, 0.01 * 2.0 / (2.0 + 1e-8), rtol=1e-12)


def test_linear_regime_is_affine():
    """With large positive biases every ReLU is active and the net is the product
    of its affine maps."""
    params = M.init_params(4, 3, hidden=5, seed=3)
    params = [(W * (1e-3 if 0 < l < 3 else 1.0), b + (100.0 if l < 3 else 0.0))
              for l, (W, b) in enumerate(params)]
    X = np.random.default_rng(1).uniform(-1, 1, (6, 4))
    Y, _ = M.forward(params, X)
    A = np.eye(4)
    c = np.zeros(4)
    for W, b in params:
        A, c = W @ A, W @ c + b
    assert np.allclose(Y, X @ A.T + c, rtol=1e-12, atol=1e-10)
