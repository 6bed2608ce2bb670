"""HSS representation (Section 3.1, Figures 1-2) built from explicit blocks.

TEST INFRASTRUCTURE ONLY.  For a symmetric matrix A in cluster order and
the postorder tree of ``cluster``:

* leaf i:      D_i = A(I_i, I_i);
* every non-root node i: a row interpolative decomposition of its
  off-diagonal block row, A(I_i, I_i^c) ~= U_i A(J_i, I_i^c), where the
  skeleton J_i is a subset of the rows and U_i(J_i, :) = I.  For a leaf the
  rows are I_i; for a parent they are the children's skeletons J_c1, J_c2,
  so U_i = diag(U_c1, U_c2) Utilde_i is nested as in Section 3.1 and only
  Utilde_i is stored.  Since A is symmetric, V_i = U_i.
* non-leaf i with children a, b: B_ab = A(J_a, J_b) and B_ba = B_ab^T.

The interpolative decomposition is a Householder QR with column pivoting
of the transposed block row: at each step the pivot is the remaining
column of largest 2-norm (norms recomputed, ties to the lowest index); the
numerical rank is the number of pivots with |R_jj| > eps * |R_11| (and
> eps_abs); T = R11^{-1} R12 by back substitution; the rows not in the
skeleton are represented as T^T times the skeleton rows.

This explicit construction is what the randomized algorithm the paper
uses (its ref. [2], Martinsson 2011) approximates from samples A R; the
generators are not unique (they depend on the pivot order), so only
densified matrices, residuals and accuracies are compared with another
implementation.
"""
from __future__ import annotations

import numpy as np


def back_substitute(R: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve R X = B for upper-triangular R (k x k)."""
    k = R.shape[0]
    X = np.array(B, dtype=np.float64, copy=True)
    for i in range(k - 1, -1, -1):
        if i + 1 < k:
            X[i] -= R[i, i + 1:] @ X[i + 1:]
        X[i] /= R[i, i]
    return X


def pivoted_qr(A: np.ndarray, eps: float, eps_abs: float = 0.0):
    """Householder QR with column pivoting, stopped at the numerical rank.

    Returns (k, piv, R) where A[:, piv] = Q R and R is k x ncols (upper
    trapezoidal in its first k columns).
    """
    A = np.array(A, dtype=np.float64, copy=True)
    nr, nc = A.shape
    piv = np.arange(nc)
    r11 = None
    k = 0
    for j in range(min(nr, nc)):
        norms = np.sqrt((A[j:, j:] ** 2).sum(axis=0))
        p = j + int(np.argmax(norms))
        nrm = norms[p - j]
        if r11 is None:
            r11 = nrm
        if not (nrm > eps * r11) or not (nrm > eps_abs):
            break
        if p != j:
            A[:, [j, p]] = A[:, [p, j]]
            piv[[j, p]] = piv[[p, j]]
        v = A[j:, j].copy()
        alpha = -nrm if v[0] >= 0 else nrm
        v[0] -= alpha
        vn = np.sqrt(v @ v)
        if vn > 0:
            v /= vn
            A[j:, j:] -= 2.0 * np.outer(v, v @ A[j:, j:])
        A[j, j] = alpha
        A[j + 1:, j] = 0.0
        k = j + 1
    return k, piv, A[:k, :]


def row_id(M: np.ndarray, eps: float, eps_abs: float = 0.0):
    """Row interpolative decomposition M ~= U M[J, :].

    Returns (J, U) with J the skeleton rows (positions into M) and U of
    shape (m, k), U[J] = I.
    """
    m = M.shape[0]
    k, piv, R = pivoted_qr(M.T, eps, eps_abs)
    T = back_substitute(R[:, :k], R[:, k:]) if k > 0 else np.zeros((0, m))
    U = np.zeros((m, k))
    U[piv[:k], np.arange(k)] = 1.0
    U[piv[k:], :] = T.T
    return piv[:k].copy(), U


class HSS:
    """Generators of a symmetric HSS matrix on a postorder tree."""

    def __init__(self, tree_arrays):
        self.t = tree_arrays
        nn = len(tree_arrays["begin"])
        self.D = [None] * nn
        self.U = [None] * nn      # Utilde (leaf: |I| x k; parent: (k_a+k_b) x k)
        self.J = [None] * nn      # skeleton, global (permuted-order) row indices
        self.B = [None] * nn      # B_ab at the parent of (a, b)

    @property
    def root(self):
        return len(self.t["begin"]) - 1

    def ranks(self):
        return [None if u is None else u.shape[1] for u in self.U]

    def max_rank(self):
        return max([u.shape[1] for u in self.U if u is not None] or [0])

    def memory_entries(self):
        """Entries stored in D_i, U_i and B_ij (V_i = U_i, B_ji = B_ij^T)."""
        s = 0
        for x in self.D + self.U + self.B:
            if x is not None:
                s += x.size
        return s


def build_explicit(A: np.ndarray, tree_arrays, eps: float, eps_abs: float = 0.0) -> HSS:
    """HSS of the symmetric matrix A (already in cluster order)."""
    t = tree_arrays
    H = HSS(t)
    n = A.shape[0]
    nn = len(t["begin"])
    for i in range(nn):
        b, e = int(t["begin"][i]), int(t["end"][i])
        l, r = int(t["left"][i]), int(t["right"][i])
        if l < 0:
            rows = np.arange(b, e)
            H.D[i] = A[np.ix_(rows, rows)].copy()
        else:
            rows = np.concatenate([H.J[l], H.J[r]])
            H.B[i] = A[np.ix_(H.J[l], H.J[r])].copy()
        if t["parent"][i] >= 0:
            cols = np.concatenate([np.arange(0, b), np.arange(e, n)])
            M = A[np.ix_(rows, cols)]
            Jloc, U = row_id(M, eps, eps_abs)
            H.J[i] = rows[Jloc]
            H.U[i] = U
    return H


def full_bases(H: HSS):
    """Expanded nested bases U_i (|I_i| x k_i) for every non-root node."""
    t = H.t
    Uf = [None] * len(t["begin"])
    for i in range(len(t["begin"])):
        if t["parent"][i] < 0:
            continue
        l, r = int(t["left"][i]), int(t["right"][i])
        if l < 0:
            Uf[i] = H.U[i]
        else:
            ka = Uf[l].shape[1]
            top = Uf[l] @ H.U[i][:ka]
            bot = Uf[r] @ H.U[i][ka:]
            Uf[i] = np.vstack([top, bot])
    return Uf


def densify(H: HSS) -> np.ndarray:
    """The dense matrix an HSS represents."""
    t = H.t
    n = int(t["end"][H.root]) if len(t["end"]) else 0
    Uf = full_bases(H)
    M = np.zeros((n, n))
    for i in range(len(t["begin"])):
        b, e = int(t["begin"][i]), int(t["end"][i])
        l, r = int(t["left"][i]), int(t["right"][i])
        if l < 0:
            M[b:e, b:e] = H.D[i]
        else:
            lb, le = int(t["begin"][l]), int(t["end"][l])
            rb, re = int(t["begin"][r]), int(t["end"][r])
            blk = Uf[l] @ H.B[i] @ Uf[r].T
            M[lb:le, rb:re] = blk
            M[rb:re, lb:le] = blk.T
    return M
