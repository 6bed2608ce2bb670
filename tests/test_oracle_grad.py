"""Pins of the oracle's held-out-loss gradient against central finite
differences (step 1e-4) of the oracle's own dense loss -- an independent
route: the difference quotient uses only the loss (solve + product), never
the gradient formulas."""
import numpy as np

import synth
from oracle import grad, prep


def _data(n=160, m=60, d=6, seed=4):
    X, y, Xt, yt, _, _ = synth.mixture(n, d, 4, 0.7, seed, m)
    Z, Zt, _, _ = prep.standardize(X, Xt)
    return Z, Zt, y, yt


def test_grad_h_lambda_match_central_differences():
    X, Xt, y, yt = _data()
    h, lam = 1.1, 0.7
    L, dh, dlam, dX = grad.loss_and_grad(X, Xt, y, yt, h, lam)
    assert abs(L - grad.loss(X, Xt, y, yt, h, lam)) <= 1e-12 * L
    fd_h = grad.central_fd(lambda t: grad.loss(X, Xt, y, yt, t, lam), h, 1e-4)
    fd_l = grad.central_fd(lambda t: grad.loss(X, Xt, y, yt, h, t), lam, 1e-4)
    assert abs(dh - fd_h) <= 1e-6 * max(1.0, abs(dh))
    assert abs(dlam - fd_l) <= 1e-6 * max(1.0, abs(dlam))


def test_grad_x_matches_central_differences():
    X, Xt, y, yt = _data()
    h, lam = 0.9, 0.5
    _, _, _, dX = grad.loss_and_grad(X, Xt, y, yt, h, lam)
    rng = np.random.default_rng(0)
    for _ in range(8):
        p, q = int(rng.integers(0, X.shape[0])), int(rng.integers(0, X.shape[1]))

        def f(v):
            Xm = X.copy()
            Xm[p, q] = v
            return grad.loss(Xm, Xt, y, yt, h, lam)

        fd = grad.central_fd(f, X[p, q], 1e-4)
        assert abs(dX[p, q] - fd) <= 1e-6 * max(1.0, np.abs(dX).max())


def test_grad_zero_at_perfect_fit_direction():
    """If the held-out targets equal the model's own predictions the loss
    and every gradient component vanish."""
    X, Xt, y, _ = _data()
    from oracle import solve, kernel
    alpha = solve.krr_dense(X, y, 1.0, 1.0)
    yt = kernel.kernel_product(Xt, X, 1.0, alpha)[:, 0]
    L, dh, dlam, dX = grad.loss_and_grad(X, Xt, y, yt, 1.0, 1.0)
    assert L < 1e-20 and abs(dh) < 1e-9 and abs(dlam) < 1e-9 and np.abs(dX).max() < 1e-9


def test_grad_single_training_point_closed_form():
    """n = 1: K = [1], alpha = y / (1 + lambda), prediction k' alpha with
    k'_k = exp(-|x'_k - x|^2 / (2 h^2)); the loss and its three derivatives
    written out by hand."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 4))
    Xt = rng.standard_normal((5, 4))
    y = np.array([0.7])
    yt = rng.standard_normal(5)
    h, lam = 1.3, 0.4
    L, dh, dlam, dX = grad.loss_and_grad(x, Xt, y, yt, h, lam)
    D = ((Xt - x) ** 2).sum(1)
    k = np.exp(-D / (2 * h * h))
    a = y[0] / (1 + lam)
    g = k * a - yt
    assert abs(L - 0.5 * (g @ g)) <= 1e-14
    # dL/dlambda = sum_k g_k k_k d(alpha)/dlambda, d(alpha)/dlambda = -y / (1 + lambda)^2
    assert abs(dlam - (g @ k) * (-y[0] / (1 + lam) ** 2)) <= 1e-13
    # dL/dh = sum_k g_k alpha dk_k/dh, dk/dh = k D / h^3
    assert abs(dh - (g * a * k * D / h ** 3).sum()) <= 1e-13
    # dL/dx = sum_k g_k alpha dk_k/dx, dk/dx = k (x'_k - x) / h^2
    ref = ((g * a * k)[:, None] * (Xt - x)).sum(0) / h ** 2
    assert np.abs(dX[0] - ref).max() <= 1e-13
