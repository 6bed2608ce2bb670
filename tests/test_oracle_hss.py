"""Pins of the oracle's explicit HSS (Section 3.1): pivoted QR against
LAPACK, exact recovery of known-rank matrices, exactness at a tiny
tolerance, the one-leaf special case, and O(eps) error of the densified
matrix."""
import numpy as np
import scipy.linalg as sl

import synth
from oracle import cluster, hss, kernel, prep


def test_pivoted_qr_matches_lapack():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(30, 12)) * np.logspace(0, -3, 12)
    k, piv, R = hss.pivoted_qr(A, 1e-15)
    Q2, R2, p2 = sl.qr(A, pivoting=True)
    assert k == 12
    assert np.array_equal(piv, p2)
    np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(R2)), rtol=1e-12)


def test_row_id_exact_rank():
    rng = np.random.default_rng(4)
    for k in (1, 3, 7):
        M = rng.normal(size=(20, k)) @ rng.normal(size=(k, 35))
        J, U = hss.row_id(M, 1e-10)
        assert len(J) == k
        np.testing.assert_allclose(U[J], np.eye(k), atol=0)
        np.testing.assert_allclose(U @ M[J], M, atol=1e-11 * np.abs(M).max())


def _setup(n, leaf, h=1.0, lam=1.0, seed=1):
    X, *_ = synth.mixture(n, 8, 4, 0.7, seed)
    Z, *_ = prep.standardize(X)
    Z32 = Z.astype(np.float32)
    perm, tree, _ = cluster.two_means_tree(Z32, leaf, seed)
    Xp = Z32[perm].astype(float)
    A = kernel.kernel_matrix(Xp, Xp, h) + lam * np.eye(n)
    return A, tree.arrays()


def test_tiny_tolerance_is_exact():
    A, t = _setup(300, 32)
    H = hss.build_explicit(A, t, 1e-14)
    np.testing.assert_allclose(hss.densify(H), A, atol=1e-12)


def test_single_leaf_is_dense():
    A, t = _setup(100, 128)
    assert len(t["begin"]) == 1
    H = hss.build_explicit(A, t, 1e-2)
    assert np.array_equal(hss.densify(H), A)


def test_error_is_order_eps():
    A, t = _setup(600, 32)
    for eps in (1e-2, 1e-4, 1e-6):
        H = hss.build_explicit(A, t, eps)
        err = np.linalg.norm(hss.densify(H) - A) / np.linalg.norm(A)
        assert err < 10 * eps
        assert H.max_rank() < 600


def _leaves(t):
    return [v for v in range(len(t["begin"])) if t["left"][v] < 0]


def test_rank_one_limit_h_to_infinity():
    """K -> all ones as h -> infinity (Eq. (1)): every off-diagonal block has
    rank exactly 1, so every node's rank is 1, each skeleton is the node's
    first row (pivoting takes the first of equal columns), and the memory is
    the leaves' D blocks plus one column per leaf, two entries per inner
    non-root node and one B entry per inner node."""
    _, t = _setup(400, 32)
    n, lam = 400, 2.0
    A = np.ones((n, n)) + lam * np.eye(n)
    H = hss.build_explicit(A, t, 1e-8)
    root = len(t["begin"]) - 1
    ranks = H.ranks()
    assert all(ranks[v] == 1 for v in range(root))
    leaves = _leaves(t)
    assert all(H.J[v].tolist() == [t["begin"][v]] for v in leaves)
    inner = [v for v in range(len(t["begin"])) if t["left"][v] >= 0]
    m = [int(t["end"][v] - t["begin"][v]) for v in leaves]
    expect = sum(x * x for x in m) + sum(m) + 2 * (len(inner) - 1) + len(inner)
    assert H.memory_entries() == expect
    np.testing.assert_allclose(hss.densify(H), A, rtol=0, atol=1e-13)


def test_rank_zero_limit_h_to_zero():
    """K -> I as h -> 0: the off-diagonal blocks vanish, every rank is 0 and
    the HSS is its leaves' diagonal blocks."""
    _, t = _setup(300, 32)
    n, lam = 300, 0.5
    A = (1.0 + lam) * np.eye(n)
    H = hss.build_explicit(A, t, 1e-8)
    assert H.max_rank() == 0
    m = [int(t["end"][v] - t["begin"][v]) for v in _leaves(t)]
    assert H.memory_entries() == sum(x * x for x in m)
    assert np.array_equal(hss.densify(H), A)
