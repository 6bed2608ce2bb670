"""Pins of the oracle's recursive two-means (Sections 4.2-4.3): a worked
example, the Lloyd fixed point on tiny inputs checked by brute force, the
tree invariants, and the integer bounds of the quantization."""
import os

import numpy as np
import pytest

import synth
from oracle import cluster

GOLD = os.path.join(os.path.dirname(__file__), "golden", "two_means_1d.txt")


def _tree_ok(perm, tree, n, leaf):
    a = tree.arrays()
    assert np.array_equal(np.sort(perm), np.arange(n))
    root = tree.n_nodes - 1
    assert a["begin"][root] == 0 and a["end"][root] == n and a["parent"][root] == -1
    for i in range(tree.n_nodes):
        l, r = a["left"][i], a["right"][i]
        if l < 0:
            assert 0 < a["end"][i] - a["begin"][i] <= leaf or n == 0
        else:
            assert a["end"][i] - a["begin"][i] > leaf
            assert l < i and r < i and l < r                     # postorder
            assert a["begin"][l] == a["begin"][i] and a["end"][r] == a["end"][i]
            assert a["end"][l] == a["begin"][r]
            assert a["parent"][l] == i and a["parent"][r] == i
            assert a["level"][l] == a["level"][i] + 1


def test_golden_two_groups():
    lines = {l.split(":")[0]: l.split(":")[1] for l in open(GOLD) if ":" in l and not l.startswith("#")}
    pts = np.array(lines["points"].split(), float)[:, None].astype(np.float32)
    leaf = int(lines["leaf"])
    g1, g2 = [set(float(v) for v in s.split()) for s in lines["groups"].split("|")]
    for seed in range(20):
        perm, tree, _ = cluster.two_means_tree(pts, leaf, seed)
        assert tree.n_nodes == 3
        a = tree.arrays()
        first = set(pts[perm[a["begin"][0]:a["end"][0]], 0].tolist())
        second = set(pts[perm[a["begin"][1]:a["end"][1]], 0].tolist())
        assert {frozenset(first), frozenset(second)} == {frozenset(g1), frozenset(g2)}


def test_lloyd_fixed_point_brute_force():
    """The final split of every non-halved node is a Lloyd fixed point: each
    point is no farther from its own centre than from the other (tie to
    group 0) and each centre is the rounded mean of its group."""
    rng = np.random.default_rng(0)
    for trial in range(40):
        n = int(rng.integers(3, 13))
        X = rng.normal(size=(n, 2)).astype(np.float32)
        q, _ = cluster.quantize(X)
        labels, it, halved = cluster.split_node(q, seed=trial, begin=0)
        if halved or it == cluster.MAX_ITER:
            continue
        c = [None, None]
        for g in (0, 1):
            pts = q[labels == g]
            c[g] = np.array([(2 * int(s) + len(pts)) // (2 * len(pts)) for s in pts.sum(0)])
        for i in range(n):
            d0 = sum((int(q[i, k]) - int(c[0][k])) ** 2 for k in range(2))
            d1 = sum((int(q[i, k]) - int(c[1][k])) ** 2 for k in range(2))
            assert labels[i] == (0 if d0 <= d1 else 1)


def test_quantization_bounds():
    """Every squared distance between points or centres of the hull, summed
    over all n points, stays below 2^63; the exponent is the largest with
    that property."""
    for n, d in ((1000, 8), (65536, 8), (7, 1), (3000, 54)):
        X = np.zeros((n, d), np.float32)
        X[0, 0] = -3.75
        X[-1, -1] = 2.5
        k = cluster.quant_exponent(X)
        qmax = abs(np.rint(-3.75 * 2.0 ** k))
        assert n * d * (2 * qmax) ** 2 <= 2 ** 63
        assert n * d * (4 * qmax) ** 2 > 2 ** 63 / 16     # one more bit would not fit


def test_tree_invariants_mixture():
    X, *_ = synth.mixture(3000, 8, 8, 0.7, 3)
    X = X.astype(np.float32)
    for leaf in (16, 64, 128):
        perm, tree, st = cluster.two_means_tree(X, leaf, 7)
        _tree_ok(perm, tree, 3000, leaf)


def test_identical_points_are_halved():
    X = np.ones((40, 3), np.float32)
    perm, tree, st = cluster.two_means_tree(X, 8, 1)
    _tree_ok(perm, tree, 40, 8)
    assert np.array_equal(perm, np.arange(40))
    a = tree.arrays()
    assert sorted((a["end"] - a["begin"])[a["left"] < 0].tolist()) == [5] * 8


def test_deterministic_and_seeded():
    X, *_ = synth.mixture(2000, 5, 6, 0.7, 8)
    X = X.astype(np.float32)
    p1, _, _ = cluster.two_means_tree(X, 50, 3)
    p2, _, _ = cluster.two_means_tree(X, 50, 3)
    p3, _, _ = cluster.two_means_tree(X, 50, 4)
    assert np.array_equal(p1, p2)
    assert not np.array_equal(p1, p3)


def test_natural_tree():
    perm, tree = cluster.natural_tree(100, 16)
    _tree_ok(perm, tree, 100, 16)


def test_nonfinite_rejected():
    X = np.zeros((10, 2), np.float32)
    X[3, 1] = np.nan
    with pytest.raises(ValueError):
        cluster.two_means_tree(X, 4, 0)


def test_second_seed_boundary_rule_worked_example():
    """The second representative is the first row whose inclusive prefix sum
    of squared distances exceeds the target.  Hand-worked: weights
    [0, 4, 1, 9] have prefix sums [0, 4, 5, 14]; targets 0..3 land in row 1,
    target 4 (exactly on the boundary) in row 2, targets 5..13 in row 3.
    The zero-weight row (the first representative itself) is never drawn."""
    w = np.array([0, 4, 1, 9], dtype=np.uint64)
    got = [cluster.pick_by_weight(w, t) for t in range(14)]
    assert got == [1, 1, 1, 1, 2] + [3] * 9
    # a zero weight in the middle is skipped as well
    assert [cluster.pick_by_weight(np.array([2, 0, 3], np.uint64), t) for t in range(5)] == [0, 0, 2, 2, 2]


def test_second_seed_frequencies_follow_squared_distance():
    """Section 4.3 draws the second point with probability growing with its
    distance from the first; the oracle reads this as the squared distance
    (k-means++ weight).  Over 20000 seeds the draws on five 1-D points must
    follow D^2 / sum D^2 given the first point (chi-square, p > 1e-3); the
    plain-distance weights are rejected by the same test."""
    from scipy.stats import chisquare
    q = np.array([[0], [1], [3], [6], [10]], dtype=np.int64)
    counts = np.zeros((5, 5), dtype=np.int64)
    for seed in range(20000):
        f, s, total = cluster.seed_pair(q, seed, 0)
        assert s is not None and s != f
        counts[f, s] += 1
    for f in range(5):
        n_f = counts[f].sum()
        assert n_f > 3000                          # the first point is uniform
        others = [j for j in range(5) if j != f]
        d2 = np.array([float((q[j, 0] - q[f, 0]) ** 2) for j in others])
        p = chisquare(counts[f, others], n_f * d2 / d2.sum()).pvalue
        assert p > 1e-3, (f, counts[f], p)
        d1 = np.sqrt(d2)
        assert chisquare(counts[f, others], n_f * d1 / d1.sum()).pvalue < 1e-6


def test_kd_split_worked_examples():
    """k-d split (Section 4.3): coordinate of maximum spread, split at its
    mean; 100 x smaller side < larger side falls back to the median."""
    # spread x = 10 > spread y = 5: split x at its mean 4.4 -> {0, 1, 2} | {9, 10}
    P = np.array([[0, 0], [1, 5], [2, 1], [9, 2], [10, 3]], np.float32)
    perm, tree = cluster.kd_tree(P, 3)
    a = tree.arrays()
    assert tree.n_nodes == 3 and sorted(perm[a["begin"][0]:a["end"][0]].tolist()) == [0, 1, 2]
    # equal spreads: the lower coordinate; a point exactly at the mean goes first
    Q = np.array([[0, 4], [2, 0], [4, 2]], np.float32)   # x: 0,2,4 (mean 2), y: 4,0,2 (mean 2)
    assert cluster.kd_split(cluster.quantize(Q)[0]).tolist() == [0, 0, 1]
    # 200 zeros and one outlier: the mean split is 200 | 1 (100 * 1 < 200), so the
    # median split puts the first floor(201 / 2) = 100 rows of the tie first
    R = np.zeros((201, 1), np.float32)
    R[150, 0] = 1000.0
    lab = cluster.kd_split(cluster.quantize(R)[0])
    assert lab[:100].tolist() == [0] * 100 and lab[100:].sum() == 101
    # all points identical: halves
    assert cluster.kd_split(np.zeros((5, 3), np.int64)).tolist() == [0, 0, 1, 1, 1]


def test_pca_direction_matches_lapack_eigenvector():
    """The power iteration of pca_direction reaches the top eigenvector of
    the node's covariance (numpy.linalg.eigh, a library routine) when the
    spectrum has a clear gap; the split separates the points by the sign of
    their projection relative to the mean."""
    rng = np.random.default_rng(5)
    for d in (2, 5, 8):
        X = (rng.standard_normal((400, d)) * np.r_[3.0, np.linspace(1.2, 0.5, d - 1)]).astype(np.float32)
        q, _ = cluster.quantize(X)
        mu, v = cluster.pca_direction(q)
        qf = q.astype(np.float64)
        C = np.cov(qf.T, bias=True)
        w, U = np.linalg.eigh(C)
        u = U[:, -1] * np.sign(U[np.argmax(np.abs(U[:, -1])), -1])
        assert np.allclose(v, u, atol=1e-9), (d, v, u)
        lab = cluster.pca_split(q)
        p = (qf - qf.mean(0)) @ u
        assert np.array_equal(lab, (p > 0).astype(np.int8)) or np.min(np.abs(p)) < 1e-6 * np.abs(p).max()
    # identical points: no direction, halves
    assert cluster.pca_direction(np.ones((4, 3), np.int64))[1] is None
    assert cluster.pca_split(np.ones((4, 3), np.int64)).tolist() == [0, 0, 1, 1]


@pytest.mark.parametrize("name", ["kd_tree", "pca_tree"])
def test_kd_and_pca_tree_invariants(name):
    X = synth.mixture(3000, 6, 8, 0.7, 9)[0].astype(np.float32)
    perm, tree = getattr(cluster, name)(X, 64)
    _tree_ok(perm, tree, 3000, 64)


def test_natural_order_halves():
    perm, tree = cluster.natural_tree(1000, 64)
    _tree_ok(perm, tree, 1000, 64)
    a = tree.arrays()
    sizes = (a["end"] - a["begin"])[a["left"] < 0]
    assert sizes.max() - sizes.min() <= 1 and np.array_equal(perm, np.arange(1000))
