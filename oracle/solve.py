"""Dense solve, prediction and accuracy (Algorithm 1 steps 2-4, Eq. (2)).

TEST INFRASTRUCTURE ONLY.

* ``cholesky``: right-looking Cholesky A = L L^T, written out, FP64.
* ``spd_solve``: two triangular substitutions with that factor.  Above
  ``LAPACK_ABOVE`` rows the factor and substitutions use LAPACK through
  NumPy/SciPy instead (same mathematics; the hand-written loop is checked
  against LAPACK on small systems).
* ``krr_dense``: w = (K + lambda I)^{-1} y with K from ``kernel``.
* ``predict``: decision values K(X', X) w; labels sign(.), with sign(0) = +1
  (the paper leaves sign(0) open).
* ``accuracy``: the fraction of test labels predicted correctly (Eq. (2)).
* ``residual``: ||(K + lambda I) a - y|| / ||y|| per right-hand side.
"""
from __future__ import annotations

import numpy as np

from . import kernel

LAPACK_ABOVE = 1536


def cholesky(A: np.ndarray) -> np.ndarray:
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        piv = A[j, j]
        if not piv > 0.0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        ljj = np.sqrt(piv)
        L[j, j] = ljj
        col = A[j + 1:, j] / ljj
        L[j + 1:, j] = col
        A[j + 1:, j + 1:] -= np.outer(col, col)
    return L


def forward_sub(L, B):
    X = np.array(B, dtype=np.float64, copy=True)
    for i in range(L.shape[0]):
        if i:
            X[i] -= L[i, :i] @ X[:i]
        X[i] /= L[i, i]
    return X


def backward_sub_t(L, B):
    """Solve L^T X = B."""
    X = np.array(B, dtype=np.float64, copy=True)
    n = L.shape[0]
    for i in range(n - 1, -1, -1):
        if i + 1 < n:
            X[i] -= L[i + 1:, i] @ X[i + 1:]
        X[i] /= L[i, i]
    return X


def spd_solve(A, Y):
    A = np.asarray(A, dtype=np.float64)
    if A.shape[0] > LAPACK_ABOVE:
        import scipy.linalg as sl
        c = sl.cho_factor(A, lower=True)
        return sl.cho_solve(c, Y)
    L = cholesky(A)
    return backward_sub_t(L, forward_sub(L, Y))


def krr_dense(X, y, h, lam):
    K = kernel.kernel_matrix(X, X, h)
    K[np.diag_indices_from(K)] += lam
    return spd_solve(K, y)


def predict(Xt, X, w, h):
    return kernel.kernel_product(Xt, X, h, w)


def sign_pm1(v):
    return np.where(np.asarray(v) >= 0, 1.0, -1.0)


def accuracy(pred_labels, true_labels) -> float:
    p = np.asarray(pred_labels).ravel()
    t = np.asarray(true_labels).ravel()
    return float(np.count_nonzero(p == t)) / max(t.size, 1)


def residual(X, h, lam, a, y, rows=None):
    """||(K + lambda I) a - y|| / ||y|| for each column (all rows, or a subset
    ``rows`` when only sampled rows are affordable)."""
    a = np.asarray(a, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if a.ndim == 1:
        a, y = a[:, None], y[:, None]
    Ka = kernel.kernel_product(X, X, h, a, rows=rows)
    if rows is None:
        r = Ka + lam * a - y
        yy = y
    else:
        r = Ka + lam * a[rows] - y[rows]
        yy = y[rows]
    return np.linalg.norm(r, axis=0) / np.linalg.norm(yy, axis=0)
