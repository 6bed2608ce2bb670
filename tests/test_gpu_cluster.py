"""Bit-exact parity of the GPU recursive two-means ordering (Sections
4.2-4.3) with the oracle, through the C-ABI, on the same FP32 inputs."""
import numpy as np
import pytest
import torch

import synth
from oracle import cluster, prep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import paper_1803_10274_gb300 as K
    return K


@pytest.fixture(scope="module")
def ctx(K):
    c = K.Context()
    yield c
    c.close()


def _check(K, ctx, X32, leaf, seed):
    perm_o, tree_o, _ = cluster.two_means_tree(X32, leaf, seed)
    perm_g, tree_g = K.krr_cluster(ctx, torch.from_numpy(X32).cuda(), leaf, seed)
    assert np.array_equal(perm_g.cpu().numpy(), perm_o)
    a = tree_o.arrays()
    for k in ("begin", "end", "left", "right", "parent", "level"):
        assert np.array_equal(tree_g[k], a[k]), k


@pytest.mark.parametrize("n,d,comp,leaf,seed", [(1000, 8, 4, 64, 1),       # the small plain workload
                                                (5000, 3, 7, 16, 5),
                                                (3333, 54, 7, 100, 9),
                                                (20000, 8, 16, 128, 2),
                                                (1500, 128, 5, 64, 3)])
def test_mixture_bit_exact(K, ctx, n, d, comp, leaf, seed):
    X, *_ = synth.mixture(n, d, comp, 0.7, seed)
    Z, *_ = prep.standardize(X)
    _check(K, ctx, Z.astype(np.float32), leaf, seed)


def test_image_like_d784_bit_exact(K, ctx):
    """MNIST-shaped rows: d = 784, most coordinates exactly zero."""
    X = synth.image_like(1000, 3)[0].astype(np.float32)
    _check(K, ctx, X, 128, 4)
    X = synth.image_like(3000, 5)[0].astype(np.float32)   # 12 blocks of 256 rows, leaf 256
    _check(K, ctx, X, 256, 6)


@pytest.mark.parametrize("n,d,comp,leaf,seed", [(2500, 64, 5, 100, 11),   # 4 coordinates per lane
                                                (1700, 200, 6, 64, 12),    # 8
                                                (1300, 300, 4, 128, 13),   # 16
                                                (2100, 700, 5, 128, 14),   # 32, shared memory above 48 KB
                                                (1100, 1024, 3, 64, 15)])  # the largest d
def test_wide_rows_bit_exact(K, ctx, n, d, comp, leaf, seed):
    """Rows of 64 or more coordinates (a warp per point, each coordinate
    read once per Lloyd pass), ragged n: blocks of one node, blocks across
    nodes, and partial last blocks."""
    X, *_ = synth.mixture(n, d, comp, 0.7, seed)
    Z, *_ = prep.standardize(X)
    _check(K, ctx, Z.astype(np.float32), leaf, seed)


def test_full_size_bit_exact(K, ctx):
    """The 65536-point, 8-feature, leaf-128 ordering the benchmark uses."""
    X, *_ = synth.mixture(65536, 8, 16, 0.7, 2)
    Z, *_ = prep.standardize(X)
    _check(K, ctx, Z.astype(np.float32), 128, 2)


def test_degenerate_inputs(K, ctx):
    _check(K, ctx, np.ones((300, 4), np.float32), 16, 3)          # all identical: halves
    X = np.repeat(np.arange(5, dtype=np.float32)[:, None], 60, axis=0)  # heavy duplicates
    _check(K, ctx, X, 7, 4)
    _check(K, ctx, np.zeros((1, 2), np.float32), 1, 0)            # single point
    rng = np.random.default_rng(0)
    _check(K, ctx, rng.normal(size=(129, 2)).astype(np.float32), 128, 8)   # one split


def test_nonfinite_rejected(K, ctx):
    X = np.zeros((50, 2), np.float32)
    X[7, 1] = np.inf
    with pytest.raises(K.KRRError):
        K.krr_cluster(ctx, torch.from_numpy(X).cuda(), 8, 0)
