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
