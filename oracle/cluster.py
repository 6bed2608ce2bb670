"""Recursive two-means (2MN) ordering and the HSS cluster tree.

TEST INFRASTRUCTURE ONLY.  Follows the paper's Section 4.2 (split the
points into two groups, make each group contiguous, recurse on both
groups while a group is larger than the leaf size) and Section 4.3
("Recursive two-means": pick one point at random, pick a second one with
probability growing with its distance from the first, then alternate
nearest-representative assignment and centre updates until no point
changes side).  Nodes are numbered in postorder, as in Figure 2.

The paper fixes no arithmetic, so this oracle takes the following
reading, chosen so that any correct implementation reaches the same
permutation bit for bit:

1. Coordinates are quantized once: q = round_half_even(x * 2^k) with the
   largest k for which every squared distance between points (or centres)
   inside the hull, summed over all n points, stays below 2^63.
   Distances, sums and centres are then exact 64-bit integers.
2. The centre of a group is floor((2 * sum q + cnt) / (2 * cnt)) per
   coordinate (the mean rounded half up).
3. Seeding of the node covering rows [b, b + m): Philox4x64-10 words
   (w0, w1) at counter (b, m, 0, 0) (``rng.cluster_words``).  First
   representative: row b + floor(w0 * m / 2^64).  Second: drawn with
   probability proportional to the SQUARED distance to the first (the
   k-means++ weight; the paper says "proportional to the distance",
   squared is taken so the draw stays in exact integers): target =
   floor(w1 * total / 2^64), pick the first row whose inclusive prefix sum
   of squared distances exceeds target.  If all points coincide (total 0)
   the node is split into halves.
4. A point goes to group 0 iff its squared distance to centre 0 is <= its
   squared distance to centre 1.
5. Iterate: assign; stop if no label changed (the first assignment always
   counts as a change); stop if a group is empty; recompute both centres;
   stop after MAX_ITER centre updates.
6. If a group is empty at the end, split at floor(m / 2) in the current
   order (the NP rule of Section 4.3).
7. Stable partition, group 0 first; children in that order; recurse while
   m > leaf.
"""
from __future__ import annotations

import math
import sys

import numpy as np

from .rng import cluster_words, mulhi64

MAX_ITER = 100


def quant_exponent(X32: np.ndarray) -> int:
    """k such that q = rint(x * 2^k) keeps every sum of squared distances < 2^63."""
    X = np.asarray(X32, dtype=np.float32)
    n, d = X.shape
    L = (4 * d * n - 1).bit_length()          # ceil(log2(4 d n))
    t = (63 - L) // 2
    maxabs = float(np.max(np.abs(X))) if X.size else 0.0
    if maxabs == 0.0:
        return 0
    e = math.frexp(maxabs)[1]                 # maxabs < 2^e
    return t - e


def quantize(X32: np.ndarray):
    X = np.asarray(X32, dtype=np.float32)
    if not np.all(np.isfinite(X)):
        raise ValueError("non-finite coordinate")
    k = quant_exponent(X)
    q = np.rint(X.astype(np.float64) * math.ldexp(1.0, k)).astype(np.int64)
    return q, k


def _centre(qs: np.ndarray) -> np.ndarray:
    cnt = qs.shape[0]
    s = qs.sum(axis=0, dtype=np.int64)
    return (2 * s + cnt) // (2 * cnt)


def pick_by_weight(weights, target: int) -> int:
    """Index of the first entry whose inclusive prefix sum of the
    non-negative integer weights exceeds target (0 <= target < total), so
    entry j is picked for exactly weights[j] of the total target values."""
    prefix = np.cumsum(np.asarray(weights, dtype=np.uint64), dtype=np.uint64)
    return int(np.searchsorted(prefix, np.uint64(target), side="right"))


def seed_pair(q: np.ndarray, seed: int, begin: int):
    """The two starting representatives of the node with rows q (m x d)
    that starts at row ``begin``: (first, second, total).  The first is
    uniform over the rows; the second is drawn with probability
    proportional to the squared distance to the first (reading 3 above);
    second is None when every row coincides with the first (total 0)."""
    m = q.shape[0]
    w0, w1 = cluster_words(seed, begin, m)
    first = mulhi64(w0, m)
    dist = ((q - q[first]) ** 2).sum(axis=1)
    du = dist.astype(np.uint64)
    total = int(du.sum(dtype=np.uint64))
    if total == 0:
        return first, None, 0
    return first, pick_by_weight(du, mulhi64(w1, total)), total


def split_node(q: np.ndarray, seed: int, begin: int):
    """Two-means labels (0/1, int8) of the m rows q (m x d) of one node.

    Returns (labels, n_centre_updates, halved).
    """
    m = q.shape[0]
    first, second, total = seed_pair(q, seed, begin)
    halves = (np.arange(m) >= m // 2).astype(np.int8)
    if total == 0:
        return halves, 0, True
    c0 = q[first].copy()
    c1 = q[second].copy()

    labels = None
    it = 0
    while True:
        d0 = ((q - c0) ** 2).sum(axis=1)
        d1 = ((q - c1) ** 2).sum(axis=1)
        new = (d0 > d1).astype(np.int8)
        changed = labels is None or bool(np.any(new != labels))
        labels = new
        if not changed:
            break
        cnt1 = int(labels.sum())
        cnt0 = m - cnt1
        if cnt0 == 0 or cnt1 == 0:
            break
        c0 = _centre(q[labels == 0])
        c1 = _centre(q[labels == 1])
        it += 1
        if it == MAX_ITER:
            break
    cnt1 = int(labels.sum())
    if cnt1 == 0 or cnt1 == m:
        return halves, it, True
    return labels, it, False


class Tree:
    """Binary cluster tree in postorder (Figure 2 numbering).

    begin/end: row range in the permuted order; left/right: child ids or
    -1 for a leaf; parent: -1 for the root; level: depth (root 0).
    """

    def __init__(self):
        self.begin, self.end, self.left, self.right, self.parent, self.level = ([] for _ in range(6))

    def add(self, b, e, l, r, lev):
        i = len(self.begin)
        self.begin.append(b); self.end.append(e); self.left.append(l)
        self.right.append(r); self.parent.append(-1); self.level.append(lev)
        if l >= 0:
            self.parent[l] = i
            self.parent[r] = i
        return i

    def arrays(self):
        return {k: np.asarray(getattr(self, k), dtype=np.int32)
                for k in ("begin", "end", "left", "right", "parent", "level")}

    @property
    def n_nodes(self):
        return len(self.begin)


def two_means_tree(X32: np.ndarray, leaf: int, seed: int):
    """Recursive two-means ordering.

    Returns (perm, tree, stats): perm[new] = old row index; tree in
    postorder; stats holds the per-node centre-update counts.
    """
    if leaf < 1:
        raise ValueError("leaf must be >= 1")
    q, k = quantize(X32)
    n = q.shape[0]
    perm = np.arange(n, dtype=np.int64)
    tree = Tree()
    iters = {}

    def build(b, e, lev):
        m = e - b
        if m <= leaf:
            return tree.add(b, e, -1, -1, lev)
        labels, it, halved = split_node(q[b:e], seed, b)
        order = np.concatenate([np.nonzero(labels == 0)[0], np.nonzero(labels == 1)[0]])
        q[b:e] = q[b:e][order]
        perm[b:e] = perm[b:e][order]
        c0 = int(np.count_nonzero(labels == 0))
        l = build(b, b + c0, lev + 1)
        r = build(b + c0, e, lev + 1)
        nid = tree.add(b, e, l, r, lev)
        iters[nid] = (it, halved)
        return nid

    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 4 * n // max(leaf, 1) + 1000))
    try:
        if n > 0:
            build(0, n, 0)
    finally:
        sys.setrecursionlimit(old)
    return perm.astype(np.int32), tree, {"centre_updates": iters, "quant_exp": k}


def _build_tree(q, leaf, split):
    """Recursive divisive ordering shared by the KD and PCA readings:
    split(q_rows) -> int8 labels (0 = first child); a split with an empty
    side becomes halves.  Stable partition, postorder numbering."""
    n = q.shape[0]
    q = q.copy()
    perm = np.arange(n, dtype=np.int64)
    tree = Tree()

    def build(b, e, lev):
        m = e - b
        if m <= leaf:
            return tree.add(b, e, -1, -1, lev)
        labels = split(q[b:e])
        c1 = int(labels.sum())
        if c1 == 0 or c1 == m:
            labels = (np.arange(m) >= m // 2).astype(np.int8)
        order = np.concatenate([np.nonzero(labels == 0)[0], np.nonzero(labels == 1)[0]])
        q[b:e] = q[b:e][order]
        perm[b:e] = perm[b:e][order]
        c0 = int(np.count_nonzero(labels == 0))
        l = build(b, b + c0, lev + 1)
        r = build(b + c0, e, lev + 1)
        return tree.add(b, e, l, r, lev)

    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 4 * n // max(leaf, 1) + 1000))
    try:
        if n > 0:
            build(0, n, 0)
    finally:
        sys.setrecursionlimit(old)
    return perm.astype(np.int32), tree


KD_UNBALANCED = 100  # mean split rejected when 100 * |smaller side| < |larger side|


def kd_split(q: np.ndarray) -> np.ndarray:
    """k-d tree split of one node (Section 4.3, "K-d tree"): the coordinate
    of maximum spread (read as max - min of the quantized coordinates;
    lowest index on ties), split at its mean (a point goes to the first
    child iff its value is <= the mean, i.e. q * m <= sum q, exact in
    integers); if 100 * |smaller side| < |larger side| the split moves to
    the median: the floor(m / 2) smallest values go first, ties by row
    order.  All points identical: halves."""
    m = q.shape[0]
    spread = q.max(axis=0) - q.min(axis=0)
    k = int(np.argmax(spread))                  # first maximum
    if spread[k] == 0:
        return (np.arange(m) >= m // 2).astype(np.int8)
    col = q[:, k]
    tot = int(col.sum())
    labels = np.array([0 if int(v) * m <= tot else 1 for v in col], dtype=np.int8)
    c1 = int(labels.sum())
    c0 = m - c1
    if KD_UNBALANCED * min(c0, c1) < max(c0, c1):
        rank = np.lexsort((np.arange(m), col))   # by value, then row order
        labels = np.ones(m, dtype=np.int8)
        labels[rank[: m // 2]] = 0
    return labels


PCA_POWER_ITERS = 64


def pca_direction(q: np.ndarray):
    """First principal direction of the node's quantized points (Section
    4.3, "Principal component analysis"), as a fixed sequence of IEEE FP64
    operations (no fused multiply-add), so every implementation that follows
    it gets the same bits:
      mu_a  = double(sum_i q_ia) / m
      C_ab  = double(sum_i q_ia q_ib) / m - mu_a * mu_b   (sums exact in int64)
      v     = e_0 ... then PCA_POWER_ITERS times w = C v (sum over b in
              order), v = w / sqrt(sum_a w_a^2); stop early if w = 0;
      sign: the entry of largest magnitude (lowest index on ties) positive.
    Returns (mu, v); v is None when C is zero (all points identical)."""
    m, d = q.shape
    s = [int(q[:, a].sum()) for a in range(d)]
    mu = [float(s[a]) / float(m) for a in range(d)]
    C = [[0.0] * d for _ in range(d)]
    zero = True
    for a in range(d):
        for b in range(d):
            sab = int(np.dot(q[:, a], q[:, b]))           # exact: |sum| < 2^63 by the quantization
            C[a][b] = float(sab) / float(m) - mu[a] * mu[b]
            zero = zero and C[a][b] == 0.0
    if zero:
        return mu, None
    v = [1.0] + [0.0] * (d - 1)
    for _ in range(PCA_POWER_ITERS):
        w = [0.0] * d
        for a in range(d):
            acc = 0.0
            for b in range(d):
                acc = acc + C[a][b] * v[b]
            w[a] = acc
        nrm = 0.0
        for a in range(d):
            nrm = nrm + w[a] * w[a]
        if nrm == 0.0:
            break
        nrm = math.sqrt(nrm)
        v = [w[a] / nrm for a in range(d)]
    big = 0
    for a in range(1, d):
        if abs(v[a]) > abs(v[big]):
            big = a
    if v[big] < 0:
        v = [-x for x in v]
    return mu, v


def pca_split(q: np.ndarray) -> np.ndarray:
    """PCA split of one node: a point goes to the first child iff its
    projection onto the principal direction, relative to the mean, is
    <= 0: p_i = sum_a (double(q_ia) - mu_a) * v_a, summed over a in order."""
    m, d = q.shape
    mu, v = pca_direction(q)
    if v is None:
        return (np.arange(m) >= m // 2).astype(np.int8)
    p = np.zeros(m)
    for a in range(d):
        p = p + (q[:, a].astype(np.float64) - mu[a]) * v[a]
    return (p > 0).astype(np.int8)


def kd_tree(X32: np.ndarray, leaf: int):
    """Recursive k-d tree ordering (KD, Section 4.3).  Returns (perm, tree)."""
    if leaf < 1:
        raise ValueError("leaf must be >= 1")
    q, _ = quantize(X32)
    return _build_tree(q, leaf, kd_split)


def pca_tree(X32: np.ndarray, leaf: int):
    """Recursive principal-direction ordering (PCA, Section 4.3).  Returns
    (perm, tree)."""
    if leaf < 1:
        raise ValueError("leaf must be >= 1")
    q, _ = quantize(X32)
    return _build_tree(q, leaf, pca_split)


def natural_tree(n: int, leaf: int):
    """No preprocessing (NP, Section 4.3): natural order, halves (+-1)."""
    tree = Tree()

    def build(b, e, lev):
        if e - b <= leaf:
            return tree.add(b, e, -1, -1, lev)
        mid = b + (e - b) // 2
        l = build(b, mid, lev + 1)
        r = build(mid, e, lev + 1)
        return tree.add(b, e, l, r, lev)

    if n > 0:
        build(0, n, 0)
    return np.arange(n, dtype=np.int32), tree
