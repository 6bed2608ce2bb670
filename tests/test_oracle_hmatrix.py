"""Pins of the oracle's H-matrix sampler (Section 3.2, the H matrix
representation: strong admissibility, low-rank far blocks by adaptive cross
approximation) against facts that do not depend on it: exact reproduction
of low-rank matrices, the cross-interpolation property, every entry covered
by exactly one block, eta = 0 equal to the dense kernel product, box
distances worked out by hand."""
import numpy as np
import pytest

from oracle import cluster, hmatrix, kernel


def _two_means_order(n, d, leaf, seed):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-4, 4, size=(6, d))
    X = centres[rng.integers(0, 6, n)] + 0.6 * rng.standard_normal((n, d))
    X32 = X.astype(np.float32)
    perm, tree, _ = cluster.two_means_tree(X32, leaf, seed)
    return X32[perm].astype(np.float64), tree.arrays()


# ------------------------------------------------------------ boxes and admissibility
def test_box_distance_and_diameter_by_hand():
    lo = np.array([[0.0, 0.0], [2.0, 0.0], [0.5, 0.5], [3.0, 4.0]])
    hi = np.array([[1.0, 1.0], [3.0, 1.0], [2.5, 0.7], [4.0, 5.0]])
    assert hmatrix.diam(lo, hi, 0) == pytest.approx(np.sqrt(2.0))
    assert hmatrix.dist(lo, hi, 0, 1) == pytest.approx(1.0)          # apart along x only
    assert hmatrix.dist(lo, hi, 0, 2) == 0.0                         # overlapping
    assert hmatrix.dist(lo, hi, 0, 3) == pytest.approx(np.hypot(2.0, 3.0))
    assert hmatrix.dist(lo, hi, 1, 0) == hmatrix.dist(lo, hi, 0, 1)  # symmetric
    # min(diam) = sqrt(2) against dist 1
    assert not hmatrix.admissible(lo, hi, 0, 1, 1.0)
    assert hmatrix.admissible(lo, hi, 0, 1, 1.5)
    assert not hmatrix.admissible(lo, hi, 0, 2, 1e9)                 # touching boxes never are


def test_partition_of_a_four_leaf_tree_by_hand():
    # postorder: leaves 0, 1 under 2; leaves 3, 4 under 5; root 6
    t = {"begin": np.array([0, 2, 0, 4, 6, 4, 0]), "end": np.array([2, 4, 4, 6, 8, 8, 8]),
         "left": np.array([-1, -1, 0, -1, -1, 3, 2]), "right": np.array([-1, -1, 1, -1, -1, 4, 5])}
    # 1-D boxes: leaves at [0,1], [2,3], [10,11], [12,13]
    lo = np.array([[0.0], [2.0], [0.0], [10.0], [12.0], [10.0], [0.0]])
    hi = np.array([[1.0], [3.0], [3.0], [11.0], [13.0], [13.0], [13.0]])
    near, far = hmatrix.block_partition(t, lo, hi, 1.0)
    # (2, 5) and (5, 2): diam 3 each, dist 7; the leaves: neighbours at
    # distance 1 with diam 1 are admissible, a leaf with itself is not
    assert far == [(0, 1), (1, 0), (2, 5), (5, 2), (3, 4), (4, 3)]
    assert near == [(0, 0), (1, 1), (3, 3), (4, 4)]
    near, far = hmatrix.block_partition(t, lo, hi, 0.5)
    assert far == [(2, 5), (5, 2)]
    assert near == [(0, 0), (0, 1), (1, 0), (1, 1), (3, 3), (3, 4), (4, 3), (4, 4)]


@pytest.mark.parametrize("eta", [0.5, 1.0, 2.0])
def test_partition_covers_every_entry_exactly_once(eta):
    X, t = _two_means_order(400, 2, 16, 3)
    lo, hi = hmatrix.node_boxes(X, t)
    near, far = hmatrix.block_partition(t, lo, hi, eta)
    b, e = t["begin"], t["end"]
    cover = np.zeros((len(X), len(X)), dtype=np.int32)
    for tt, s in near + far:
        cover[b[tt]:e[tt], b[s]:e[s]] += 1
    assert np.all(cover == 1)
    assert all(t["left"][tt] < 0 and t["left"][s] < 0 for tt, s in near)
    assert all(hmatrix.admissible(lo, hi, tt, s, eta) for tt, s in far)
    assert not any(hmatrix.admissible(lo, hi, tt, s, eta) for tt, s in near)
    assert len(far) > 0


def test_boxes_contain_their_points():
    X, t = _two_means_order(300, 3, 20, 4)
    lo, hi = hmatrix.node_boxes(X, t)
    for v in range(len(t["begin"])):
        P = X[t["begin"][v]:t["end"][v]]
        assert np.all(P >= lo[v]) and np.all(P <= hi[v])
        assert np.any(P == lo[v], axis=0).all() and np.any(P == hi[v], axis=0).all()


# ------------------------------------------------------------ cross approximation
def _aca_of(A, eps, max_rank=None):
    return hmatrix.aca(lambda i: A[i], lambda j: A[:, j], A.shape[0], A.shape[1], eps, max_rank)


@pytest.mark.parametrize("r", [1, 3, 7])
def test_aca_reproduces_a_low_rank_matrix(r):
    rng = np.random.default_rng(r)
    A = rng.standard_normal((40, r)) @ rng.standard_normal((r, 30))
    U, V, rows, cols = _aca_of(A, 1e-13)
    assert U.shape[1] <= r + 1   # the last step may add a rounding-size term
    assert np.linalg.norm(A - U @ V.T) <= 1e-11 * np.linalg.norm(A)
    assert len(set(rows)) == len(rows) and len(set(cols)) == len(cols)


def test_aca_interpolates_the_pivot_rows_and_columns():
    X, _ = _two_means_order(200, 3, 200, 5)
    A = kernel.kernel_matrix(X[:90], X[110:], 1.5)
    U, V, rows, cols = _aca_of(A, 1e-4)
    k = U.shape[1]
    assert 0 < k < min(A.shape)
    R = A - U @ V.T
    scale = np.abs(A).max()
    assert np.abs(R[rows, :]).max() <= 1e-12 * scale
    assert np.abs(R[:, cols]).max() <= 1e-12 * scale


def test_aca_of_a_zero_block_has_rank_zero():
    A = np.zeros((12, 9))
    U, V, rows, cols = _aca_of(A, 1e-8)
    assert U.shape == (12, 0) and V.shape == (9, 0) and rows == [] and cols == []


def test_aca_rank_cap():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((20, 20))
    U, V, _, _ = _aca_of(A, 1e-15, max_rank=5)
    assert U.shape[1] == 5
    U, V, _, _ = _aca_of(A, 1e-15)
    assert U.shape[1] == 20 and np.linalg.norm(A - U @ V.T) <= 1e-10 * np.linalg.norm(A)


def test_aca_error_on_well_separated_kernel_blocks():
    """Gaussian-kernel blocks between two separated clusters: the stopping
    rule's estimate tracks the true error (within 10 eps relative), and the
    rank is no larger than the SVD's at a 100 times smaller tolerance."""
    rng = np.random.default_rng(7)
    P = rng.standard_normal((150, 4)) * 0.5
    Q = rng.standard_normal((120, 4)) * 0.5 + np.array([4.0, 0, 0, 0])
    for h, eps in ((1.0, 1e-6), (2.0, 1e-8)):
        A = kernel.kernel_matrix(P, Q, h)
        U, V, _, _ = hmatrix.aca(lambda i: A[i], lambda j: A[:, j], 150, 120, eps)
        err = np.linalg.norm(A - U @ V.T)
        assert err <= 10 * eps * np.linalg.norm(A)
        s = np.linalg.svd(A, compute_uv=False)
        assert U.shape[1] <= np.count_nonzero(s > 0.01 * eps * s[0]) + 1


# ------------------------------------------------------------ the H-matrix product
def test_eta_zero_is_the_dense_product():
    X, t = _two_means_order(350, 3, 24, 6)
    rng = np.random.default_rng(1)
    R = rng.standard_normal((350, 5))
    H = hmatrix.HMatrix(X, 1.2, t, eta=0.0, eps=1e-8)
    assert H.far == []
    S = kernel.kernel_product(X, X, 1.2, R)
    assert np.allclose(H.matvec(R), S, rtol=0, atol=1e-12 * np.abs(S).max())
    assert np.allclose(H.matvec(R, lam=3.0), S + 3.0 * R, rtol=0, atol=1e-12 * np.abs(S).max())
    # the same-leaf mask of the sampling product
    leaf = np.full(350, -1, np.int32)
    for v in range(len(t["begin"])):
        if t["left"][v] < 0:
            leaf[t["begin"][v]:t["end"][v]] = v
    Sm = kernel.kernel_product(X, X, 1.2, R, leaf, leaf)
    assert np.allclose(H.matvec(R, skip_same_leaf=True), Sm, rtol=0, atol=1e-12 * np.abs(S).max())


@pytest.mark.parametrize("eta,eps", [(1.0, 1e-6), (2.0, 1e-9)])
def test_h_product_within_the_cross_tolerance(eta, eps):
    X, t = _two_means_order(600, 3, 24, 8)
    rng = np.random.default_rng(2)
    R = rng.standard_normal((600, 4))
    H = hmatrix.HMatrix(X, 1.0, t, eta=eta, eps=eps)
    assert len(H.far) > 0 and H.near_entries() < 600 * 600
    S = kernel.kernel_product(X, X, 1.0, R)
    Sa = kernel.kernel_product(X, X, 1.0, np.abs(R))
    err = np.abs(H.matvec(R) - S)
    # each far block is within 10 eps in the Frobenius norm; per entry this
    # is loose, so the bound is taken against the absolute product
    assert np.all(err <= 100 * eps * Sa.max())
