"""Pins of the oracle's dense path (Algorithm 1 steps 2-4, Eq. (2)):
hand-written Cholesky against LAPACK, the solve against a library solve,
prediction / accuracy on a worked example."""
import numpy as np

import synth
from oracle import kernel, prep, solve


def test_cholesky_matches_lapack():
    rng = np.random.default_rng(0)
    B = rng.normal(size=(60, 60))
    A = B @ B.T + 60 * np.eye(60)
    np.testing.assert_allclose(solve.cholesky(A), np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    Y = rng.normal(size=(60, 3))
    np.testing.assert_allclose(solve.spd_solve(A, Y), np.linalg.solve(A, Y), rtol=1e-10)


def test_not_spd_raises():
    import pytest
    with pytest.raises(np.linalg.LinAlgError):
        solve.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_krr_dense_residual_and_accuracy():
    X, y, Xt, yt, _, _ = synth.mixture(1000, 8, 4, 0.7, 1, 200)
    w = solve.krr_dense(X, y, 1.0, 1.0)
    res = solve.residual(X, 1.0, 1.0, w, y)
    assert res[0] < 1e-12
    acc = solve.accuracy(solve.sign_pm1(solve.predict(Xt, X, w, 1.0)), yt)
    assert acc > 0.75


def test_accuracy_and_sign_worked_example():
    assert solve.accuracy([1, -1, 1, 1], [1, 1, 1, -1]) == 0.5
    assert list(solve.sign_pm1([0.0, -0.0, -1e-300, 2.0])) == [1.0, 1.0, -1.0, 1.0]


def test_standardize():
    rng = np.random.default_rng(1)
    X = rng.normal(3.0, 2.0, size=(500, 4))
    X[:, 2] = 7.0
    Z, Zt, m, s = prep.standardize(X, X[:5])
    np.testing.assert_allclose(Z.mean(0), 0, atol=1e-12)
    np.testing.assert_allclose(Z[:, [0, 1, 3]].std(0), 1, rtol=1e-12)
    assert np.all(Z[:, 2] == 0)
    np.testing.assert_allclose(Zt, Z[:5])


def test_dense_large_route_equals_hand_cholesky():
    """The in-place 64-bit LAPACK route used for the 65536-point golden
    solve gives the hand-written Cholesky's solution (n below LAPACK_ABOVE)."""
    import synth
    X, y, *_ = synth.mixture(900, 8, 4, 0.7, 7)
    a = solve.krr_dense(X, y, 1.0, 1.0)
    b = solve.krr_dense_large(X, y, 1.0, 1.0)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_one_vs_all_targets_and_argmax_worked_example():
    """One-vs-all (Section 2 after Algorithm 1): one +1 per row; argmax with
    the lowest class on ties; the literal |.| confidence differs from the
    signed one on a point that is strongly "not class 0"."""
    Y = solve.one_vs_all_targets([2, 0, 1, 2], 3)
    assert Y.tolist() == [[-1, -1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]]
    dec = np.array([[0.2, 0.9, -0.1],
                    [0.5, 0.5, 0.1],      # tie: lowest index
                    [-3.0, 0.4, 0.2],     # signed -> 1, absolute -> 0
                    [-0.1, -0.2, -0.3]])
    assert solve.predict_classes(dec).tolist() == [1, 0, 1, 0]
    assert solve.predict_classes(dec, absolute=True).tolist() == [1, 0, 0, 2]


def test_two_classes_reduce_to_the_sign_rule():
    """With c = 2 the one-vs-all targets are y and -y, so w(1) = -w(0) and
    the signed argmax is the binary rule sign(w^T K'(i)) with sign(0) = +1
    (class 0 <-> label +1) of Algorithm 1 step 4."""
    import synth
    X, y, Xt, yt, comp, comp_t = synth.mixture(300, 4, 2, 0.7, 11, 120)
    cls = (comp % 2).astype(np.int32)          # class 0 <-> label +1
    W = solve.krr_dense(X, solve.one_vs_all_targets(cls, 2), 1.0, 1.0)
    dec = solve.predict(Xt, X, W, 1.0)
    w = solve.krr_dense(X, np.where(cls == 0, 1.0, -1.0), 1.0, 1.0)
    lab = solve.sign_pm1(solve.predict(Xt, X, w, 1.0)[:, 0])
    assert np.array_equal(solve.predict_classes(dec), np.where(lab > 0, 0, 1))
