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


def test_adamw_decay_with_zero_gradient():
    """With a zero gradient Adam's moments stay zero, so the step is the pure
    decoupled decay: W <- (1 - lr wd) W, biases unchanged."""
    import numpy as np
    from oracle import mlp as omlp
    rng = np.random.default_rng(0)
    params = [(rng.normal(size=(4, 3)), rng.normal(size=4)), (rng.normal(size=(2, 4)),
                                                              rng.normal(size=2))]
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    opt = mlp.Adam(params, lr=1e-2, weight_decay=0.5)
    new = opt.step(params, zeros)
    for (W, b), (W1, b1) in zip(params, new):
        np.testing.assert_allclose(W1, (1 - 1e-2 * 0.5) * W, rtol=1e-15)
        np.testing.assert_array_equal(b1, b)


def test_blend_weight_minimises_a_linear_residual_on_the_segment():
    import numpy as np
    from oracle import mlp as omlp
    rng = np.random.default_rng(2)
    A = rng.normal(size=(30, 12))
    f = rng.normal(size=30)
    for trial in range(20):
        u0, u1 = rng.normal(size=12), rng.normal(size=12)
        r0, r1 = A @ u0 - f, A @ u1 - f
        alpha = mlp.blend_weight(r0, r1)
        grid = np.linspace(0.0, 1.0, 20001)
        res = [np.linalg.norm(A @ ((1 - a) * u0 + a * u1) - f) for a in grid]
        best = grid[int(np.argmin(res))]
        assert abs(alpha - best) <= 1e-4, (alpha, best)


# --- the degree projection of the learned correction (smoothing) -----------

@pytest.mark.parametrize("order,q", [(1, 0), (2, 1), (3, 1), (4, 2), (4, 0), (6, 3)])
def test_degree_projection_pins(order, q):
    """Pinned by what an L2 projection is: polynomials of degree <= q in each
    direction are reproduced, a Legendre mode of degree q + 1 along any axis
    is removed, the map is idempotent, and in 1-D it equals weighted least
    squares on the monomials x^0..x^q (numpy lstsq) with the GL weights."""
    m = order + 1
    x, w = np.polynomial.legendre.leggauss(m)
    P = mlp.degree_projector(order, q)
    # 1-D: weighted least squares with a monomial basis (independent route)
    V = np.vander(x, q + 1, increasing=True)
    sw = np.sqrt(w)[:, None]
    rng = np.random.default_rng(order * 10 + q)
    f = rng.normal(size=m)
    coef, *_ = np.linalg.lstsq(sw * V, sw[:, 0] * f, rcond=None)
    np.testing.assert_allclose(P @ f, V @ coef, rtol=0, atol=1e-13)
    np.testing.assert_allclose(P @ P, P, rtol=0, atol=1e-13)
    # 3-D: tensor-product polynomials of degree <= q are kept
    gx, gy, gz = np.meshgrid(x, x, x, indexing="ij")        # (i, j, k) = (x, y, z)
    poly = (1.0 + gx ** q) * (0.5 - gy ** max(q - 1, 0)) * (2.0 + gz)
    if q == 0:
        poly = np.full_like(gx, 1.7)
    Y = np.stack([poly.transpose(2, 1, 0).reshape(-1), 2.0 * poly.transpose(2, 1, 0).reshape(-1)])
    Y = Y.reshape(-1, 1)                                     # 2 variables, one column
    np.testing.assert_allclose(mlp.project_degree(Y, order, 3, q), Y, rtol=0, atol=1e-12)
    # a Legendre mode of degree q + 1 along y alone is removed
    if q + 1 <= order:
        Lq = np.polynomial.legendre.legval(gy, [0] * (q + 1) + [1.0])
        Z = (Lq * (1.0 + gx ** min(q, 1))).transpose(2, 1, 0).reshape(-1, 1)
        np.testing.assert_allclose(mlp.project_degree(Z, order, 3, q), 0.0, rtol=0, atol=1e-12)
    # idempotent on random data, also in 2-D
    R = rng.normal(size=(3 * m ** 2, 4))
    R1 = mlp.project_degree(R, order, 2, q)
    np.testing.assert_allclose(mlp.project_degree(R1, order, 2, q), R1, rtol=0, atol=1e-12)


def test_degree_projection_catches_a_wrong_axis_order():
    """Planted mistake: projecting only along one axis (or with the degree
    taken as q + 1) leaves the degree-(q + 1) mode in place."""
    order, q = 3, 1
    m = order + 1
    x, _ = np.polynomial.legendre.leggauss(m)
    gx, gy, gz = np.meshgrid(x, x, x, indexing="ij")
    Z = np.polynomial.legendre.legval(gz, [0, 0, 1.0]).transpose(2, 1, 0).reshape(-1, 1)
    P = mlp.degree_projector(order, q)
    only_x = np.tensordot(P, Z.reshape(m, m, m, 1), axes=([1], [2])).transpose(1, 2, 0, 3)
    assert np.abs(only_x).max() > 0.1
    assert np.abs(mlp.project_degree(Z, order, 3, q + 1)).max() > 0.1
    assert np.abs(mlp.project_degree(Z, order, 3, q)).max() < 1e-12
