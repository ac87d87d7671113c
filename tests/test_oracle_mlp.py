"""Pins for the oracle's MLP (learned initial guess)."""
import numpy as np
import pytest

from oracle import mlp


def _params(rng, sizes):
    return [(rng.normal(size=(o, i)) / np.sqrt(i), rng.normal(size=o) * 0.1)
            for i, o in zip(sizes[:-1], sizes[1:])]


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    params = _params(rng, [7, 6, 5, 4])
    X = rng.normal(size=(7, 9))
    T = rng.normal(size=(4, 9))
    Y, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, Y, T)
    h = 1e-6
    for li in range(3):
        for j in range(2):
            p = params[li][j]
            g = grads[li][j]
            it = np.nditer(p, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = p[idx]
                p[idx] = old + h
                lp = mlp.loss(mlp.forward(params, X)[0], T)
                p[idx] = old - h
                lm = mlp.loss(mlp.forward(params, X)[0], T)
                p[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (li, j, idx, fd, g[idx])


def test_forward_represents_known_piecewise_linear_map():
    """relu(x) - relu(-x) = x and relu(x) + relu(-x) = |x| through two layers."""
    n = 3
    I = np.eye(n)
    W1 = np.vstack([I, -I])
    W2 = np.eye(2 * n)
    W3 = np.vstack([np.hstack([I, -I]), np.hstack([I, I])])
    params = [(W1, np.zeros(2 * n)), (W2, np.zeros(2 * n)), (W3, np.zeros(2 * n))]
    X = np.array([[1.5, -2.0], [0.0, 3.0], [-0.25, 0.5]])
    Y, _ = mlp.forward(params, X)
    np.testing.assert_allclose(Y[:n], X)
    np.testing.assert_allclose(Y[n:], np.abs(X))


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(1)
    params = _params(rng, [4, 3, 3, 2])
    grads = [(rng.normal(size=W.shape), rng.normal(size=b.shape)) for W, b in params]
    opt = mlp.Adam(params, lr=0.01, eps=1e-12)
    new = opt.step(params, grads)
    for (W, b), (Wn, bn), (gW, gb) in zip(params, new, grads):
        np.testing.assert_allclose(W - Wn, 0.01 * np.sign(gW), rtol=1e-9)
        np.testing.assert_allclose(b - bn, 0.01 * np.sign(gb), rtol=1e-9)


def test_training_reduces_loss_on_a_linear_target():
    rng = np.random.default_rng(2)
    params = _params(rng, [5, 16, 16, 3])
    A = rng.normal(size=(3, 5))
    X = rng.normal(size=(5, 200))
    T = A @ X
    opt = mlp.Adam(params, lr=3e-3)
    l0 = mlp.loss(mlp.forward(params, X)[0], T)
    for _ in range(300):
        Y, cache = mlp.forward(params, X)
        params = opt.step(params, mlp.backward(params, cache, Y, T))
    assert mlp.loss(mlp.forward(params, X)[0], T) < 0.1 * l0


def test_extrapolation_targets_vanish_for_quadratic_histories():
    rng = np.random.default_rng(3)
    a, b, c = (rng.normal(size=(7, 9, 4)) for _ in range(3))
    U = [a + b * t + c * t * t for t in (0.0, 1.0, 2.0, 3.0)]
    tg = mlp.targets(U[3], U[2], U[1], U[0], np.ones(7), elems=[0, 2, 3])
    np.testing.assert_allclose(tg, 0.0, atol=1e-12)
    X = mlp.features(U[2], U[1], U[0], (2.0 * np.ones(7), np.ones(7), 0.5 * np.ones(7)), elems=[1])
    assert X.shape == (3 * 7 * 9, 1)
    np.testing.assert_allclose(X[: 7 * 9, 0], U[2][:, :, 1].reshape(-1) / 2.0)
    # for a quadratic history the difference blocks are b + c(2t-1) and 2c
    np.testing.assert_allclose(X[7 * 9: 14 * 9, 0], (b + 3.0 * c)[:, :, 1].reshape(-1), atol=1e-12)
    np.testing.assert_allclose(X[14 * 9:, 0], (2.0 * c / 0.5)[:, :, 1].reshape(-1), atol=1e-12)
    G = mlp.apply_guess(np.zeros((7 * 9, 4)), U[2], U[1], U[0], np.ones(7))
    np.testing.assert_allclose(G, U[3], atol=1e-12)
