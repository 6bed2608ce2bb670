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
* ``one_vs_all_targets`` / ``predict_classes``: multi-class prediction by
  one-vs-all (Section 2, after Algorithm 1): c binary right-hand sides,
  the class of a test point is the argmax over c of its confidence.
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


def _lapack_mkl():
    """LAPACK of the MKL build that PyTorch links (32-bit integer interface;
    MKL computes its offsets in 64 bits, so n^2 >= 2^31 is fine)."""
    import ctypes
    import os
    import torch
    L = ctypes.CDLL(os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cpu.so"))
    i32p, P = ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p
    # Fortran interface: arguments by reference, the hidden string length last
    L.dpotrf_.argtypes = [ctypes.c_char_p, i32p, P, i32p, i32p, ctypes.c_size_t]
    L.dpotrf_.restype = None
    L.dpotrs_.argtypes = [ctypes.c_char_p, i32p, i32p, P, i32p, P, i32p, i32p, ctypes.c_size_t]
    L.dpotrs_.restype = None
    return L


def krr_dense_large(X, y, h, lam):
    """krr_dense for large n with one n x n FP64 array only: K + lambda I is
    built once and LAPACK (dpotrf, dpotrs) factors and solves it in place.
    K is symmetric, so its row-major buffer is also the column-major matrix
    LAPACK reads.  Same mathematics as krr_dense; n = 65536 needs 32 GiB of
    host memory."""
    import ctypes
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    K = kernel.kernel_matrix(X, X, h)
    K[np.diag_indices_from(K)] += lam
    L = _lapack_mkl()
    i32 = ctypes.c_int32
    nn, info = i32(n), i32(0)
    L.dpotrf_(b"L", ctypes.byref(nn), K.ctypes.data, ctypes.byref(nn), ctypes.byref(info), 1)
    if info.value != 0:
        raise np.linalg.LinAlgError("dpotrf failed (info %d)" % info.value)
    Y = np.array(np.asarray(y, dtype=np.float64).reshape(n, -1), order="F", copy=True)
    nrhs = i32(Y.shape[1])
    L.dpotrs_(b"L", ctypes.byref(nn), ctypes.byref(nrhs), K.ctypes.data, ctypes.byref(nn),
              Y.ctypes.data, ctypes.byref(nn), ctypes.byref(info), 1)
    if info.value != 0:
        raise np.linalg.LinAlgError("dpotrs failed (info %d)" % info.value)
    del K
    return np.ascontiguousarray(Y).reshape(np.shape(y))


def predict(Xt, X, w, h):
    return kernel.kernel_product(Xt, X, h, w)


def sign_pm1(v):
    return np.where(np.asarray(v) >= 0, 1.0, -1.0)


def one_vs_all_targets(cls, c: int) -> np.ndarray:
    """n x c right-hand sides: +1 in column k for the points of class k,
    -1 elsewhere (one binary classifier per class)."""
    cls = np.asarray(cls).ravel()
    Y = -np.ones((cls.size, c))
    for i in range(cls.size):
        Y[i, int(cls[i])] = 1.0
    return Y


def predict_classes(dec, absolute: bool = False) -> np.ndarray:
    """Class of each test point: the argmax over the c columns of its
    decision values (Section 2 after Algorithm 1), lowest class index on a
    tie.  The paper prints the confidence as |w(c)^T K'(i)|; read literally
    (absolute=True) a strong "not class c" counts as confidence in c, so the
    default reading takes the signed value, which is the confidence that
    the point belongs to class c.  Plain loops."""
    dec = np.asarray(dec, dtype=np.float64)
    m, c = dec.shape
    out = np.zeros(m, dtype=np.int32)
    for i in range(m):
        best, arg = None, 0
        for k in range(c):
            v = abs(dec[i, k]) if absolute else dec[i, k]
            if best is None or v > best:
                best, arg = v, k
        out[i] = arg
    return out


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
