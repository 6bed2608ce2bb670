"""The library's H-matrix block partition (krr_h_partition, host code of
the C ABI; Section 3.2, strong admissibility) against the oracle's: the
same near and far lists, in the same order, on two-means trees of several
data sets and admissibility parameters.  Needs no GPU."""
import numpy as np
import pytest

from oracle import cluster, hmatrix


@pytest.fixture(scope="module")
def K():
    import paper_1803_10274_gb300 as K
    return K


def _tree(n, d, leaf, seed, spread=4.0):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-spread, spread, size=(8, d))
    X = (centres[rng.integers(0, 8, n)] + 0.7 * rng.standard_normal((n, d))).astype(np.float32)
    perm, tree, _ = cluster.two_means_tree(X, leaf, seed)
    return X[perm].astype(np.float64), tree.arrays()


@pytest.mark.parametrize("n,d,leaf,seed", [(500, 2, 16, 1), (800, 3, 32, 2), (1200, 8, 64, 3), (300, 1, 8, 4)])
@pytest.mark.parametrize("eta", [0.0, 0.5, 1.0, 2.0])
def test_same_lists_as_the_oracle(K, n, d, leaf, seed, eta):
    X, t = _tree(n, d, leaf, seed)
    lo, hi = hmatrix.node_boxes(X, t)
    near_o, far_o = hmatrix.block_partition(t, lo, hi, eta)
    near, far = K.krr_h_partition(t["left"], t["right"], lo, hi, eta)
    assert [tuple(p) for p in near.tolist()] == [tuple(p) for p in near_o]
    assert [tuple(p) for p in far.tolist()] == [tuple(p) for p in far_o]


def test_capacity_overflow_is_retried_with_the_counts(K):
    # the binding starts at 4 n_nodes pairs; eta = 0 on a deep tree needs
    # more (only boxes of one point, diameter 0, are admissible there)
    X, t = _tree(2000, 2, 8, 5)
    lo, hi = hmatrix.node_boxes(X, t)
    near, far = K.krr_h_partition(t["left"], t["right"], lo, hi, 0.0)
    near_o, far_o = hmatrix.block_partition(t, lo, hi, 0.0)
    assert len(near) > 4 * len(t["left"])
    assert [tuple(p) for p in near.tolist()] == [tuple(p) for p in near_o]
    assert [tuple(p) for p in far.tolist()] == [tuple(p) for p in far_o]
    assert all(hmatrix.diam(lo, hi, a) == 0.0 or hmatrix.diam(lo, hi, b) == 0.0 for a, b in far_o)


def test_bad_trees_rejected(K):
    lo = np.zeros((3, 1))
    hi = np.ones((3, 1))
    with pytest.raises(K.KRRError):   # a node with one child
        K.krr_h_partition(np.array([-1, -1, 0]), np.array([-1, -1, -1]), lo, hi, 1.0)
    with pytest.raises(K.KRRError):   # a child numbered after its parent
        K.krr_h_partition(np.array([-1, 2, -1]), np.array([-1, 0, -1]), lo, hi, 1.0)
    with pytest.raises(K.KRRError):   # negative eta
        K.krr_h_partition(np.array([-1, -1, 0]), np.array([-1, -1, 1]), lo, hi, -1.0)
    with pytest.raises(ValueError):
        K.krr_h_partition(np.array([-1, -1, 0]), np.array([-1, -1, 1]), lo, hi[:2], 1.0)
