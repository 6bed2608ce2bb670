"""Gaussian kernel, Eq. (1) of the paper (Section 1; Algorithm 1 step 1):

    K_ij = exp( -||x_i - x_j||^2 / (2 h^2) ).

TEST INFRASTRUCTURE ONLY.  Difference form, FP64, sequential sum over the
d coordinates, evaluated by the plain C loops in ``csrc/oracle_kernel.c``.
"""
from __future__ import annotations

import numpy as np

from . import _clib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def kernel_matrix(Xa, Xb, h: float) -> np.ndarray:
    """Dense K(Xa, Xb) (ma x nb)."""
    Xa, Xb = _f64(Xa), _f64(Xb)
    ma, d = Xa.shape
    nb = Xb.shape[0]
    K = np.empty((ma, nb))
    _clib.lib().okrr_kernel_matrix(_clib.ptr(Xa), ma, _clib.ptr(Xb), nb, d, float(h), _clib.ptr(K))
    return K


def sqdist_matrix(Xa, Xb) -> np.ndarray:
    """Squared distances ||xa_i - xb_j||^2 (ma x nb), difference form."""
    Xa, Xb = _f64(Xa), _f64(Xb)
    ma, d = Xa.shape
    nb = Xb.shape[0]
    D = np.empty((ma, nb))
    _clib.lib().okrr_sqdist_matrix(_clib.ptr(Xa), ma, _clib.ptr(Xb), nb, d, _clib.ptr(D))
    return D


def kernel_product(Xa, Xb, h: float, R, leaf_a=None, leaf_b=None, rows=None,
                   want_abs: bool = False):
    """S = W o K(Xa, Xb) @ R without storing K.

    W_ij = 0 where leaf_a[i] == leaf_b[j] (both given), else 1.  ``rows``
    restricts the output to those rows of Xa.  With ``want_abs`` also
    returns the same product with |R|.
    """
    Xa, Xb = _f64(Xa), _f64(Xb)
    R = _f64(R)
    if R.ndim == 1:
        R = R[:, None]
    ma, d = Xa.shape
    nb, r = R.shape
    assert Xb.shape == (nb, d)
    la = lb = None
    if leaf_a is not None and leaf_b is not None:
        la = np.ascontiguousarray(leaf_a, dtype=np.int32)
        lb = np.ascontiguousarray(leaf_b, dtype=np.int32)
    rw = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nrows = ma if rw is None else rw.shape[0]
    S = np.empty((nrows, r))
    Sa = np.empty((nrows, r)) if want_abs else None
    _clib.lib().okrr_kernel_product(_clib.ptr(Xa), ma, _clib.ptr(Xb), nb, d, float(h),
                                    _clib.ptr(R), r, _clib.ptr(la), _clib.ptr(lb),
                                    _clib.ptr(rw), nrows, _clib.ptr(S), _clib.ptr(Sa))
    return (S, Sa) if want_abs else S


def num_threads() -> int:
    return int(_clib.lib().okrr_num_threads())
