"""Held-out loss of kernel ridge regression and its gradient with respect to
h, lambda and the training points, dense FP64.

TEST INFRASTRUCTURE ONLY.  The loss is the squared error of Algorithm 1's
decision values on held-out points (Section 5.3 tunes h and lambda on a
validation set; here the tuning criterion is made differentiable):

    alpha = (K + lambda I)^{-1} y,   g = K_t alpha - y_t,   L = 1/2 ||g||^2,

with K = K(X, X) and K_t = K(X_t, X) from Eq. (1).  With a = K_t^T g and
z = (K + lambda I)^{-1} a (K symmetric), differentiating alpha through the
solve gives

    dL/dlambda = -z . alpha
    dL/dh      = h^-3 [ g^T (K_t o D_t) alpha - z^T (K o D) alpha ]
    dL/dx_p    = h^-2 [ alpha_p sum_k g_k K_t[k,p] (x'_k - x_p)
                        - sum_j (z_p alpha_j + z_j alpha_p) K[p,j] (x_j - x_p) ]

where D, D_t hold squared distances (d/dh of exp(-D/(2h^2)) is K D / h^3,
d/dx_p of K[p,j] is K[p,j] (x_j - x_p) / h^2).
"""
from __future__ import annotations

import numpy as np

from . import kernel, solve


def _spd_factor_solver(A):
    """Solver for A x = b reusing one factorization of the SPD matrix A
    (LAPACK Cholesky above the size where the oracle's own loops get
    slow, as in ``solve.spd_solve``)."""
    if A.shape[0] > solve.LAPACK_ABOVE:
        import scipy.linalg as sl
        c = sl.cho_factor(A, lower=True)
        return lambda b: sl.cho_solve(c, b)
    L = solve.cholesky(A)
    return lambda b: solve.backward_sub_t(L, solve.forward_sub(L, b))


def loss(X, Xt, y, yt, h, lam):
    X = np.asarray(X, dtype=np.float64)
    alpha = solve.krr_dense(X, y, h, lam)
    g = kernel.kernel_product(Xt, X, h, alpha)[:, 0] - np.asarray(yt, dtype=np.float64)
    return 0.5 * float(g @ g)


def loss_and_grad(X, Xt, y, yt, h, lam):
    """(L, dL/dh, dL/dlambda, dL/dX) in FP64 with dense matrices."""
    X = np.asarray(X, dtype=np.float64)
    Xt = np.asarray(Xt, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    yt = np.asarray(yt, dtype=np.float64)
    n = X.shape[0]
    K = kernel.kernel_matrix(X, X, h)
    A = K + lam * np.eye(n)
    sol = _spd_factor_solver(A)
    del A
    alpha = sol(y)
    Kt = kernel.kernel_matrix(Xt, X, h)
    g = Kt @ alpha - yt
    L = 0.5 * float(g @ g)
    a = Kt.T @ g
    z = sol(a)
    dlam = -float(z @ alpha)
    D = kernel.sqdist_matrix(X, X)
    Dt = kernel.sqdist_matrix(Xt, X)
    dh = (float(g @ ((Kt * Dt) @ alpha)) - float(z @ ((K * D) @ alpha))) / h ** 3
    # dL/dX
    t1 = alpha[:, None] * (Kt.T @ (g[:, None] * Xt) - X * (Kt.T @ g)[:, None])
    KaX = K @ (alpha[:, None] * X)
    KzX = K @ (z[:, None] * X)
    Ka = K @ alpha
    Kz = K @ z
    t2 = z[:, None] * (KaX - X * Ka[:, None]) + alpha[:, None] * (KzX - X * Kz[:, None])
    dX = (t1 - t2) / h ** 2
    return L, dh, dlam, dX


def central_fd(fun, x0, step):
    """(f(x0 + step) - f(x0 - step)) / (2 step)."""
    return (fun(x0 + step) - fun(x0 - step)) / (2.0 * step)
