"""The orderings Section 4.3 compares with two-means (no preprocessing,
k-d tree, principal direction), through the C-ABI: permutation and tree
bit-exact against the oracle on the same FP32 inputs (integer k-d splits;
the principal direction in a fixed order of rounded FP64 operations), and
an HSS solve in each order meeting the residual gate against the FP64
operator."""
import numpy as np
import pytest
import torch

import synth
from oracle import cluster, prep, solve

pytestmark = pytest.mark.gpu

ORACLE = {1: lambda X, leaf: cluster.natural_tree(X.shape[0], leaf), 2: cluster.kd_tree, 3: cluster.pca_tree}


@pytest.fixture(scope="module")
def K():
    import paper_1803_10274_gb300 as K
    return K


@pytest.fixture(scope="module")
def ctx(K):
    c = K.Context()
    yield c
    c.close()


def _check(K, ctx, X32, leaf, ordering):
    perm_o, tree_o = ORACLE[ordering](X32, leaf)
    perm_g, tree_g = K.krr_order(ctx, torch.from_numpy(np.ascontiguousarray(X32)).cuda(), leaf, ordering)
    assert np.array_equal(perm_g.cpu().numpy(), perm_o)
    a = tree_o.arrays()
    for k in ("begin", "end", "left", "right", "parent", "level"):
        assert np.array_equal(tree_g[k], a[k]), k


@pytest.mark.parametrize("ordering", [1, 2, 3])
@pytest.mark.parametrize("n,d,comp,leaf,seed", [(4096, 8, 16, 128, 2), (3000, 6, 7, 64, 5), (777, 3, 4, 16, 9),
                                                (2000, 40, 5, 100, 4)])
def test_orderings_bit_exact(K, ctx, ordering, n, d, comp, leaf, seed):
    X = synth.mixture(n, d, comp, 0.7, seed)[0]
    X32 = prep.standardize(X)[0].astype(np.float32)
    _check(K, ctx, X32, leaf, ordering)


def test_kd_median_fallback_and_degenerate_nodes(K, ctx):
    """Far outliers make the mean split leave one side more than 100 times
    larger (the median split takes over); identical points are halved."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((3000, 4)).astype(np.float32)
    X[::700, 1] = 5000.0                      # a few huge values in one coordinate
    _check(K, ctx, X, 32, 2)
    _check(K, ctx, np.ones((300, 5), np.float32), 16, 2)
    _check(K, ctx, np.ones((300, 5), np.float32), 16, 3)
    _check(K, ctx, np.zeros((1, 2), np.float32), 4, 2)


def test_pca_dimension_limit(K, ctx):
    X = torch.zeros(100, 65, device="cuda")
    with pytest.raises(K.KRRError) as e:
        K.krr_order(ctx, X, 16, 3)
    assert e.value.code == 8              # KRR_ERR_NOT_IMPLEMENTED


@pytest.mark.parametrize("ordering", [1, 2, 3])
def test_hss_solve_in_each_order(K, ctx, ordering):
    n, h, lam = 4096, 1.0, 4.0
    X, y, *_ = synth.mixture(n, 8, 16, 0.7, 2)
    Z32 = prep.standardize(X)[0].astype(np.float32)
    o = K.default_options(h=h, lambda_=lam, eps_c=0.05, leaf=128, precision=K.KRR_MIXED, seed=2, ordering=ordering)
    H = K.hss_compress(ctx, torch.from_numpy(Z32).cuda(), o)
    H.factor()
    a, res = H.solve(torch.from_numpy(y[:, None].copy()).cuda(), tol=5e-4, max_refine=400)
    rho = solve.residual(Z32.astype(np.float64), h, lam, a.cpu().numpy(), y[:, None])
    assert rho.max() <= 1e-3
    H.close()
