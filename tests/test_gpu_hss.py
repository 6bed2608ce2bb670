"""End-to-end parity of the randomized HSS path (compression, ULV-type
factorization, GMRES with the HSS preconditioner, prediction) with the
FP64 oracle, through the C-ABI.

Gates (the method's targets): relative residual ||(K + lambda I) alpha - y||
/ ||y|| <= 10 eps against the oracle's FP64 operator; test accuracy within
0.5 points of the exact dense solve.  HSS generators are not unique (they
depend on the random block and pivot order), so they are never compared
entry by entry; exact special cases are."""
import numpy as np
import pytest
import torch

import synth
from oracle import kernel, prep, solve

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


def _fit(K, ctx, X32, Y, h, lam, eps_c, leaf, prec, tol, seed=1, **kw):
    o = K.default_options(h=h, lambda_=lam, eps_c=eps_c, leaf=leaf, precision=prec, seed=seed, **kw)
    H = K.hss_compress(ctx, torch.from_numpy(X32).cuda(), o)
    H.factor()
    a, res = H.solve(torch.from_numpy(np.ascontiguousarray(Y)).cuda(), tol=tol)
    return H, a.cpu().numpy(), res


def _rhs(y, n, extra, seed=3):
    return np.concatenate([y[:, None], np.random.default_rng(seed).standard_normal((n, extra))], 1)


def test_plain_small_workload(K, ctx):
    """n=1000, d=8 mixture of 4, h=1, lambda=1, leaf 64, eps=1e-6, 10
    right-hand sides, 200 test points, everything in FP64."""
    X, y, Xt, yt, _, _ = synth.mixture(1000, 8, 4, 0.7, 1, 200)
    X32, Xt32 = X.astype(np.float32), Xt.astype(np.float32)
    Y = _rhs(y, 1000, 9)
    eps = 1e-6
    H, A, res = _fit(K, ctx, X32, Y, 1.0, 1.0, eps, 64, K.KRR_FP64, 10 * eps)
    Xo = X32.astype(np.float64)
    rho = solve.residual(Xo, 1.0, 1.0, A, Y)
    assert rho.max() <= 10 * eps
    dec = H.predict(torch.from_numpy(Xt32).cuda(), torch.from_numpy(A[:, :1].copy()).cuda()).cpu().numpy()[:, 0]
    wd = solve.krr_dense(Xo, y, 1.0, 1.0)
    acc_d = solve.accuracy(solve.sign_pm1(solve.predict(Xt32.astype(np.float64), Xo, wd, 1.0)), yt)
    acc = solve.accuracy(solve.sign_pm1(dec), yt)
    assert abs(acc - acc_d) <= 0.005
    # decision values against the oracle's product with the same weights
    ref, ref_abs = kernel.kernel_product(Xt32, X32, 1.0, A[:, :1], want_abs=True)
    assert np.all(np.abs(dec - ref[:, 0]) <= 1e-10 * ref_abs[:, 0] + 1e-300)
    H.close()


def test_exact_at_tiny_tolerance(K, ctx):
    """With eps_c near round-off the HSS equals K + lambda I, so one ULV
    solve (no refinement) is the dense solve."""
    X, y, *_ = synth.mixture(600, 5, 3, 0.7, 4)
    X32 = X.astype(np.float32)
    H, A, _ = _fit(K, ctx, X32, y[:, None], 1.3, 0.5, 1e-13, 40, K.KRR_FP64, 0.0)
    wd = solve.krr_dense(X32.astype(np.float64), y, 1.3, 0.5)
    assert np.linalg.norm(A[:, 0] - wd) <= 1e-8 * np.linalg.norm(wd)
    H.close()


def test_single_leaf_is_dense_lu(K, ctx):
    X, y, *_ = synth.mixture(100, 3, 2, 0.7, 5)
    X32 = X.astype(np.float32)
    H, A, _ = _fit(K, ctx, X32, y[:, None], 1.0, 1.0, 0.1, 128, K.KRR_FP64, 0.0)
    wd = solve.krr_dense(X32.astype(np.float64), y, 1.0, 1.0)
    assert np.linalg.norm(A[:, 0] - wd) <= 1e-11 * np.linalg.norm(wd)
    H.close()


@pytest.mark.parametrize("prec,rtol", [("KRR_FP64", 1e-12), ("KRR_MIXED", 1e-6)])
def test_narrow_kernel_is_identity(K, ctx, prec, rtol):
    """h -> 0: K -> I (Eq. (1)).  On the lattice {-1, 0, 1}^6 (729 points,
    unit spacing) with h = 0.1 every off-diagonal entry is below e^-50, so
    every off-diagonal block is numerically zero (with an absolute pivot
    floor of 1e-12), every rank is 0, and one ULV solve gives
    alpha = y / (1 + lambda) (FP32 arithmetic on the mixed path)."""
    g = np.array(np.meshgrid(*([[-1.0, 0.0, 1.0]] * 6), indexing="ij")).reshape(6, -1).T
    X32 = (g + 0.01 * np.random.default_rng(2).standard_normal(g.shape)).astype(np.float32)
    y = np.random.default_rng(3).standard_normal(len(X32))
    H, A, res = _fit(K, ctx, X32, y[:, None], 0.1, 0.5, 0.05, 64, getattr(K, prec), 0.0, eps_abs=1e-12)
    assert H.stats()["max_rank"] == 0
    np.testing.assert_allclose(A[:, 0], y / 1.5, rtol=rtol)
    H.close()


def test_lambda_update_equals_recompression(K, ctx):
    """Section 5.3: changing lambda only changes the diagonal, so updating
    lambda and refactoring matches compressing at the new lambda (same
    random block, same ranks)."""
    X, y, *_ = synth.mixture(1500, 6, 4, 0.7, 6)
    X32 = X.astype(np.float32)
    Y = y[:, None]
    o = K.default_options(h=1.0, lambda_=1.0, eps_c=1e-4, leaf=64, precision=K.KRR_FP64, seed=3)
    H1 = K.hss_compress(ctx, torch.from_numpy(X32).cuda(), o)
    H1.update_lambda(2.5)
    H1.factor()
    a1, _ = H1.solve(torch.from_numpy(Y).cuda())
    o2 = K.default_options(h=1.0, lambda_=2.5, eps_c=1e-4, leaf=64, precision=K.KRR_FP64, seed=3)
    H2 = K.hss_compress(ctx, torch.from_numpy(X32).cuda(), o2)
    H2.factor()
    a2, _ = H2.solve(torch.from_numpy(Y).cuda())
    assert H1.stats()["max_rank"] == H2.stats()["max_rank"]
    np.testing.assert_allclose(a1.cpu().numpy(), a2.cpu().numpy(), rtol=1e-9, atol=1e-12)
    H1.close()
    H2.close()


def test_mixed_8192(K, ctx):
    """SUSY-shaped data (d=8, 16 components, standardized), h=1, lambda=4,
    leaf 128: mixed precision meets the residual and accuracy gates."""
    n = 8192
    X, y, Xt, yt, _, _ = synth.mixture(n, 8, 16, 0.7, 2, 1000)
    Z, Zt, _, _ = prep.standardize(X, Xt)
    Z32, Zt32 = Z.astype(np.float32), Zt.astype(np.float32)
    Y = _rhs(y, n, 9)
    tol = 1e-3
    H, A, res = _fit(K, ctx, Z32, Y, 1.0, 4.0, 0.05, 128, K.KRR_MIXED, 0.5 * tol)
    Zo = Z32.astype(np.float64)
    rho = solve.residual(Zo, 1.0, 4.0, A, Y)
    assert rho.max() <= tol
    dec = H.predict(torch.from_numpy(Zt32).cuda(), torch.from_numpy(A[:, :1].copy()).cuda()).cpu().numpy()[:, 0]
    wd = solve.krr_dense(Zo, y, 1.0, 4.0)
    acc_d = solve.accuracy(solve.sign_pm1(solve.predict(Zt32.astype(np.float64), Zo, wd, 1.0)), yt)
    assert abs(solve.accuracy(solve.sign_pm1(dec), yt) - acc_d) <= 0.005
    ref, ref_abs = kernel.kernel_product(Zt32, Z32, 1.0, A[:, :1], want_abs=True)
    assert np.all(np.abs(dec - ref[:, 0]) <= 2e-6 * ref_abs[:, 0] + 1e-9)
    H.close()


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    return {l.split(":")[0]: l.split(":", 1)[1].strip() for l in open(path) if ":" in l and not l.startswith("#")}


def test_mixed_full_size(K, ctx):
    """The 65536-point workload the benchmark times (10 right-hand sides):
    the residual gate over every row of the exact FP64 operator, and test
    accuracy within 0.5 points of the exact dense FP64 solve
    (tests/golden/dense_n65536.txt, written by the oracle alone)."""
    n = 65536
    X, y, Xt, yt, _, _ = synth.mixture(n, 8, 16, 0.7, 2, 4096)
    Z, Zt, _, _ = prep.standardize(X, Xt)
    Z32, Zt32 = Z.astype(np.float32), Zt.astype(np.float32)
    Y = _rhs(y, n, 9)
    tol = 1e-3
    H, A, res = _fit(K, ctx, Z32, Y, 1.0, 4.0, 0.05, 128, K.KRR_MIXED, 0.5 * tol, seed=2)
    rho = solve.residual(Z32.astype(np.float64), 1.0, 4.0, A, Y)
    assert rho.max() <= tol, rho
    dec = H.predict(torch.from_numpy(Zt32).cuda(), torch.from_numpy(A[:, :1].copy()).cuda()).cpu().numpy()[:, 0]
    lab = solve.sign_pm1(dec)
    g = _golden("dense_n65536.txt")
    assert int(g["n"]) == n and float(g["lambda"]) == 4.0
    acc_d = float(g["accuracy"])
    assert abs(solve.accuracy(lab, yt) - acc_d) <= 0.005
    dense_lab = np.array([1.0 if ch == "+" else -1.0 for ch in g["labels"]])
    assert np.mean(dense_lab == lab) >= 0.99          # the same decisions almost everywhere
    H.close()


def test_image_like_d784_mixed(K, ctx):
    """MNIST-shaped workload at n = 4096 (d = 784 raw pixels in [0, 1],
    one-vs-all class 5, h = 4, lambda = 10, leaf 256, eps = 1e-3): residual
    <= 10 eps against the oracle's operator and accuracy within 0.5 points
    of the dense solve."""
    X, y, Xt, yt = synth.image_like(4096, 3, m_test=500)
    X32, Xt32 = X.astype(np.float32), Xt.astype(np.float32)
    eps = 1e-3
    H, A, res = _fit(K, ctx, X32, y[:, None], 4.0, 10.0, 0.05, 256, K.KRR_MIXED, eps)
    Xo = X32.astype(np.float64)
    rho = solve.residual(Xo, 4.0, 10.0, A, y[:, None])
    assert rho.max() <= 10 * eps
    dec = H.predict(torch.from_numpy(Xt32).cuda(), torch.from_numpy(A.copy()).cuda()).cpu().numpy()[:, 0]
    wd = solve.krr_dense(Xo, y, 4.0, 10.0)
    acc_d = solve.accuracy(solve.sign_pm1(solve.predict(Xt32.astype(np.float64), Xo, wd, 4.0)), yt)
    assert abs(solve.accuracy(solve.sign_pm1(dec), yt) - acc_d) <= 0.005
    H.close()


def test_truncate_at_budget_still_preconditions(K, ctx):
    """KRR_TRUNCATE_AT_RMAX: with a sample budget far below the ranks the
    compression keeps truncated decompositions instead of failing, and the
    refined solve still reaches its tolerance (oracle residual)."""
    X, y, *_ = synth.mixture(4096, 8, 16, 0.7, 2)
    Z = prep.standardize(X)[0].astype(np.float32)
    o = K.default_options(h=1.0, lambda_=4.0, eps_c=0.05, leaf=128, r0=64, r_max=128, precision=K.KRR_MIXED)
    with pytest.raises(K.KRRError) as e:
        K.hss_compress(ctx, torch.from_numpy(Z).cuda(), o)
    assert e.value.code == 5
    o.flags = K.KRR_TRUNCATE_AT_RMAX
    H = K.hss_compress(ctx, torch.from_numpy(Z).cuda(), o)
    st = H.stats()
    assert st["truncated"] == 1 and st["samples"] == 128
    H.factor()
    a, res = H.solve(torch.from_numpy(y[:, None].copy()).cuda(), tol=1e-4, max_refine=600)
    rho = solve.residual(Z.astype(np.float64), 1.0, 4.0, a.cpu().numpy(), y[:, None])
    assert res <= 1e-4 and rho.max() <= 2e-4
    H.close()


def test_lambda_relative_tolerance(K, ctx):
    """KRR_LAMBDA_TOL (decompositions measured against lambda as well): the
    compression and the refined solve work with and without it, and the
    solve reaches its tolerance (oracle residual)."""
    X, y, *_ = synth.mixture(4096, 8, 4, 0.7, 21)
    Z = prep.standardize(X)[0].astype(np.float32)
    for flags in (0, K.KRR_LAMBDA_TOL):
        o = K.default_options(h=1.0, lambda_=1.0, eps_c=0.05, leaf=128, precision=K.KRR_MIXED, flags=flags)
        H = K.hss_compress(ctx, torch.from_numpy(Z).cuda(), o)
        H.factor()
        a, res = H.solve(torch.from_numpy(y[:, None].copy()).cuda(), tol=1e-4, max_refine=600)
        rho = solve.residual(Z.astype(np.float64), 1.0, 1.0, a.cpu().numpy(), y[:, None])
        assert res <= 1e-4 and rho.max() <= 2e-4
        H.close()


def test_argument_and_budget_errors(K, ctx):
    X = synth.mixture(3000, 8, 8, 0.7, 1)[0]
    Xd = torch.from_numpy(((X - X.mean(0)) / X.std(0)).astype(np.float32)).cuda()
    with pytest.raises(K.KRRError):
        K.hss_compress(ctx, Xd, K.default_options(lambda_=-1.0))
    with pytest.raises(K.KRRError) as e:
        K.hss_compress(ctx, Xd, K.default_options(h=1.0, lambda_=1.0, eps_c=1e-3, r0=64, r_max=128))
    assert e.value.code == 5            # KRR_ERR_RANK_BUDGET
    Xn = Xd.clone()
    Xn[5, 3] = float("nan")
    with pytest.raises(K.KRRError) as e:
        K.hss_compress(ctx, Xn, K.default_options())
    assert e.value.code == 2            # KRR_ERR_NONFINITE_INPUT


def test_handle_outliving_its_context(K):
    """An HSS handle still open when its context closes is destroyed with
    the context first; its own close (or garbage collection) afterwards is
    a no-op instead of a use of the freed context."""
    c = K.Context()
    X, y, *_ = synth.mixture(500, 4, 3, 0.7, 8)
    o = K.default_options(h=1.0, lambda_=1.0, eps_c=0.05, leaf=64, precision=K.KRR_MIXED, seed=1)
    H = K.hss_compress(c, torch.from_numpy(X.astype(np.float32)).cuda(), o)
    c.close()
    assert H.h is None
    H.close()
    del H
