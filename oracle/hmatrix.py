"""H-matrix sampler for the HSS construction (paper Section 3.2, the H
matrix representation, and Section 5.6 with its table of timing details:
an H matrix of the kernel, built with strong admissibility and low-rank
blocks from adaptive cross approximation, replaces the O(n^2) product K R
of the sampling stage).

TEST INFRASTRUCTURE ONLY.  Plain FP64 numpy, written to be checked by eye.
The paper describes this part in words only; the readings taken here:

* cluster tree: the HSS tree itself (recursive two-means, postorder, rows
  in cluster order); a node's box is the axis-aligned bounding box of its
  points.
* strong admissibility (Section 3.2: only well-separated sub-blocks are
  compressed): a pair of nodes (t, s) is admissible when the boxes are
  apart and min(diam t, diam s) <= eta * dist(t, s); diam is the box's
  diagonal, dist the Euclidean distance between the boxes.
* block partition: from (root, root), an admissible pair is a far block;
  two leaves are a near (dense) block; otherwise the pair is split into
  its children's pairs (both nodes split when both have children, else
  the inner one), depth first, left child first.
* far blocks: adaptive cross approximation with partial pivoting (the
  published ACA of Bebendorf, Numer. Math. 86 (2000); the paper names a
  "hybrid" ACA without details): start at the block's first row, take the
  largest residual entry of the row as pivot column (first on ties), the
  largest residual entry of the new column among unused rows as the next
  pivot row, stop when |u_k| |v_k| <= eps |U V^T|_F or at full rank; a
  zero residual row moves to the next unused row.
* the product: S = lambda R + sum over near blocks of K(t, s) R(s) +
  sum over far blocks of U (V^T R(s)); for the HSS sampling the near
  blocks of a leaf with itself are left out (the same-leaf mask of the
  dense sampling product).

Parity unpinned: nothing; every function has a pin in
tests/test_oracle_hmatrix.py (exact reproduction of low-rank blocks, the
cross-interpolation property, coverage of every entry by exactly one block,
eta = 0 equal to the dense product, the error on admissible kernel blocks).
"""
from __future__ import annotations

import numpy as np

from . import kernel


def node_boxes(X, tree_arrays):
    """Per node (postorder ids) the box of its rows [begin, end) of X:
    (lo, hi), each n_nodes x d."""
    X = np.asarray(X, dtype=np.float64)
    b, e = tree_arrays["begin"], tree_arrays["end"]
    nn = len(b)
    d = X.shape[1]
    lo = np.empty((nn, d))
    hi = np.empty((nn, d))
    for v in range(nn):
        P = X[b[v]:e[v]]
        lo[v] = P.min(axis=0)
        hi[v] = P.max(axis=0)
    return lo, hi


def _norm_seq(g):
    """sqrt of the sum of squares, summed coordinate by coordinate in order
    (the same rounding as a plain loop in any language)."""
    acc = 0.0
    for x in g:
        acc += float(x) * float(x)
    return float(np.sqrt(acc))


def diam(lo, hi, v):
    """Diagonal of node v's box."""
    return _norm_seq(hi[v] - lo[v])


def dist(lo, hi, t, s):
    """Euclidean distance between the boxes of nodes t and s (0 when they
    overlap or touch)."""
    gap = np.maximum(0.0, np.maximum(lo[s] - hi[t], lo[t] - hi[s]))
    return _norm_seq(gap)


def admissible(lo, hi, t, s, eta):
    """Strong admissibility: boxes apart and min(diam t, diam s) <= eta dist."""
    dd = dist(lo, hi, t, s)
    return dd > 0.0 and min(diam(lo, hi, t), diam(lo, hi, s)) <= eta * dd


def block_partition(tree_arrays, lo, hi, eta):
    """(near, far): lists of (t, s) node pairs in depth-first order."""
    left, right = tree_arrays["left"], tree_arrays["right"]
    root = len(left) - 1
    near, far = [], []

    def children(v):
        return (int(left[v]), int(right[v]))

    def build(t, s):
        if admissible(lo, hi, t, s, eta):
            far.append((t, s))
            return
        t_leaf, s_leaf = left[t] < 0, left[s] < 0
        if t_leaf and s_leaf:
            near.append((t, s))
        elif t_leaf:
            for s2 in children(s):
                build(t, s2)
        elif s_leaf:
            for t2 in children(t):
                build(t2, s)
        else:
            for t2 in children(t):
                for s2 in children(s):
                    build(t2, s2)

    build(root, root)
    return near, far


def aca(entry_row, entry_col, m, n, eps, max_rank=None):
    """Partially pivoted adaptive cross approximation of an m x n block
    given by entry_row(i) -> row i (length n) and entry_col(j) -> column j
    (length m).  Returns (U, V, rows, cols) with block ~= U V^T, U m x k,
    V n x k, and the pivot rows and columns in the order taken."""
    kmax = min(m, n) if max_rank is None else min(m, n, max_rank)
    us, vs = [], []
    rows, cols = [], []
    used_r = np.zeros(m, dtype=bool)
    used_c = np.zeros(n, dtype=bool)
    norm2 = 0.0  # |U V^T|_F^2 of the approximation so far
    i = 0
    while len(us) < kmax:
        # residual of row i
        row = np.array(entry_row(i), dtype=np.float64)
        for u, v in zip(us, vs):
            row -= u[i] * v
        used_r[i] = True
        cand = np.where(used_c, 0.0, np.abs(row))
        j = int(np.argmax(cand))
        if cand[j] == 0.0:
            # a zero residual row: the next unused row, if any
            free = np.nonzero(~used_r)[0]
            if free.size == 0:
                break
            i = int(free[0])
            continue
        v = row / row[j]
        col = np.array(entry_col(j), dtype=np.float64)
        for u2, v2 in zip(us, vs):
            col -= v2[j] * u2
        u = col
        used_c[j] = True
        rows.append(i)
        cols.append(j)
        # |S_k|^2 = |S_{k-1}|^2 + 2 sum_l (u_l . u)(v_l . v) + |u|^2 |v|^2
        cross = sum(float(np.dot(u2, u) * np.dot(v2, v)) for u2, v2 in zip(us, vs))
        uv = float(np.linalg.norm(u) * np.linalg.norm(v))
        norm2 += 2.0 * cross + uv * uv
        us.append(u)
        vs.append(v)
        if uv <= eps * np.sqrt(max(norm2, 0.0)):
            break
        cand_r = np.where(used_r, 0.0, np.abs(u))
        i2 = int(np.argmax(cand_r))
        if cand_r[i2] == 0.0:
            free = np.nonzero(~used_r)[0]
            if free.size == 0:
                break
            i2 = int(free[0])
        i = i2
    U = np.stack(us, axis=1) if us else np.zeros((m, 0))
    V = np.stack(vs, axis=1) if vs else np.zeros((n, 0))
    return U, V, rows, cols


def kernel_block_aca(X, h, tb, te, sb, se, eps, max_rank=None):
    """ACA of K(X[tb:te], X[sb:se]) with kernel entries computed on demand."""
    Xt, Xs = X[tb:te], X[sb:se]

    def erow(i):
        return kernel.kernel_matrix(Xt[i:i + 1], Xs, h)[0]

    def ecol(j):
        return kernel.kernel_matrix(Xt, Xs[j:j + 1], h)[:, 0]

    return aca(erow, ecol, te - tb, se - sb, eps, max_rank)


class HMatrix:
    """The near / far block lists with the far blocks' factors."""

    def __init__(self, X, h, tree_arrays, eta, eps, max_rank=None):
        self.X = np.asarray(X, dtype=np.float64)
        self.h = float(h)
        self.t = tree_arrays
        self.lo, self.hi = node_boxes(self.X, tree_arrays)
        self.near, self.far = block_partition(tree_arrays, self.lo, self.hi, eta)
        b, e = tree_arrays["begin"], tree_arrays["end"]
        self.factors = [kernel_block_aca(self.X, self.h, b[t], e[t], b[s], e[s], eps, max_rank)[:2]
                        for t, s in self.far]

    def matvec(self, R, lam=0.0, skip_same_leaf=False):
        """S = lam R + H R; with skip_same_leaf the near blocks (v, v) of a
        leaf with itself are left out."""
        R = np.asarray(R, dtype=np.float64)
        if R.ndim == 1:
            R = R[:, None]
        b, e = self.t["begin"], self.t["end"]
        S = lam * R.copy()
        for t, s in self.near:
            if skip_same_leaf and t == s:
                continue
            S[b[t]:e[t]] += kernel.kernel_matrix(self.X[b[t]:e[t]], self.X[b[s]:e[s]], self.h) @ R[b[s]:e[s]]
        for (t, s), (U, V) in zip(self.far, self.factors):
            S[b[t]:e[t]] += U @ (V.T @ R[b[s]:e[s]])
        return S

    def near_entries(self):
        b, e = self.t["begin"], self.t["end"]
        return int(sum((e[t] - b[t]) * (e[s] - b[s]) for t, s in self.near))

    def far_storage(self):
        """Entries of the far blocks' factors (U and V)."""
        return int(sum(U.size + V.size for U, V in self.factors))
