"""Pins of the oracle's Gaussian kernel (Eq. (1), Section 1) against what the
paper and mathematics fix: closed-form values, symmetry, unit diagonal, the
h -> 0 and h -> infinity limits (Section 1), positive definiteness of
K + lambda I, and the off-diagonal singular-value decay under two-means
ordering (Section 1, Table 1 / Figure 3)."""
import os

import numpy as np
import pytest

import synth
from oracle import cluster, kernel, prep

GOLD = os.path.join(os.path.dirname(__file__), "golden", "kernel_values.txt")


def _golden():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        h, a, b, v = [s.strip() for s in line.split("|")]
        rows.append((float(h), np.array(a.split(), float), np.array(b.split(), float), float(v)))
    return rows


@pytest.mark.parametrize("h,a,b,v", _golden())
def test_closed_form_values(h, a, b, v):
    K = kernel.kernel_matrix(a[None], b[None], h)
    assert abs(K[0, 0] - v) <= 2e-16 * max(1.0, v) * 4


def test_symmetric_unit_diagonal():
    X, *_ = synth.mixture(300, 5, 3, 0.7, 11)
    K = kernel.kernel_matrix(X, X, 0.8)
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 1.0)
    assert np.all((K > 0) & (K <= 1))


def test_limits_h():
    rng = np.random.default_rng(3)
    X = rng.integers(-50, 50, size=(64, 3)).astype(float)
    X = np.unique(X, axis=0)
    K0 = kernel.kernel_matrix(X, X, 1e-3)
    assert np.array_equal(K0, np.eye(X.shape[0]))        # h -> 0: identity
    Kinf = kernel.kernel_matrix(X, X, 1e6)
    assert np.max(np.abs(Kinf - 1.0)) < 1e-8              # h -> inf: all ones
    s = np.linalg.svd(Kinf, compute_uv=False)
    assert s[1] / s[0] < 1e-8                             # nearly rank one


def test_spd_shift():
    X, *_ = synth.mixture(400, 8, 4, 0.7, 5)
    lam = 0.5
    K = kernel.kernel_matrix(X, X, 1.0)
    ev = np.linalg.eigvalsh(K + lam * np.eye(len(X)))
    assert ev.min() >= lam - 1e-10


def test_product_matches_matrix_and_mask():
    X, *_ = synth.mixture(200, 4, 3, 0.7, 6)
    Y, *_ = synth.mixture(150, 4, 3, 0.7, 7)
    R = np.random.default_rng(1).standard_normal((150, 5))
    K = kernel.kernel_matrix(X, Y, 0.9)
    S = kernel.kernel_product(X, Y, 0.9, R)
    np.testing.assert_allclose(S, K @ R, rtol=1e-12, atol=1e-12)
    la = np.arange(200) // 17
    lb = np.arange(150) // 13
    W = (la[:, None] != lb[None, :]).astype(float)
    Sm, Sa = kernel.kernel_product(X, Y, 0.9, R, la, lb, want_abs=True)
    np.testing.assert_allclose(Sm, (W * K) @ R, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Sa, (W * K) @ np.abs(R), rtol=1e-12, atol=1e-12)
    rows = np.array([5, 0, 199])
    np.testing.assert_allclose(kernel.kernel_product(X, Y, 0.9, R, rows=rows), (K @ R)[rows], rtol=1e-12, atol=1e-12)


def _eff_rank(M, tol=0.01):
    s = np.linalg.svd(M, compute_uv=False)
    return int(np.count_nonzero(s > tol))


def test_two_means_speeds_up_offdiagonal_decay():
    """Section 1 / Table 1: with two-means order, the off-diagonal block
    K(1,2) between the root's two children has no more singular values above
    0.01 than with the natural order, and far fewer at intermediate h."""
    X, *_ = synth.mixture(1000, 8, 8, 0.7, 21)
    Z, *_ = prep.standardize(X)
    Z32 = Z.astype(np.float32)
    perm, tree, _ = cluster.two_means_tree(Z32, 500, 1)
    a = tree.arrays()
    l = a["left"][-1]
    cut = a["end"][l]
    Xo = Z32[perm].astype(float)
    Xn = Z32.astype(float)
    ranks = {}
    for h in (0.1, 1.0, 10.0):
        Kc = kernel.kernel_matrix(Xo, Xo, h)
        Kn = kernel.kernel_matrix(Xn, Xn, h)
        ranks[h] = (_eff_rank(Kc[:cut, cut:]), _eff_rank(Kn[:500, 500:]))
        assert ranks[h][0] <= ranks[h][1]
    assert ranks[1.0][0] < 0.8 * ranks[1.0][1]
