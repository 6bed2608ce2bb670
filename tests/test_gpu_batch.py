"""Batching: many independent problems (different sizes, widths h, shared
lambda) in one handle, against the oracle problem by problem."""
import numpy as np
import pytest
import torch

import synth
from oracle import cluster, kernel, prep, solve

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


def _problems(sizes, d, seed, m_test=0):
    """Standardized mixture draws, one per size; returns lists."""
    Xs, ys, Xts, yts = [], [], [], []
    for k, n in enumerate(sizes):
        X, y, Xt, yt, _, _ = synth.mixture(n, d, 4, 0.7, seed + k, m_test)
        Z, Zt, _, _ = prep.standardize(X, Xt if m_test else None)
        Xs.append(Z.astype(np.float32))
        ys.append(y)
        if m_test:
            Xts.append(Zt.astype(np.float32))
            yts.append(yt)
    return Xs, ys, Xts, yts


def _offsets(blocks):
    return np.concatenate([[0], np.cumsum([len(b) for b in blocks])]).astype(np.int64)


def _intervals(tree, lo, hi):
    """(begin, end, is_leaf) of the nodes inside rows [lo, hi), shifted by lo."""
    out = set()
    for b, e, l in zip(tree["begin"], tree["end"], tree["left"]):
        if b >= lo and e <= hi:
            out.add((int(b - lo), int(e - lo), bool(l < 0)))
    return out


@pytest.mark.parametrize("d", [8, 100])
def test_batched_clustering_is_each_problem_alone(K, ctx, d):
    sizes, leaf, seed = [300, 1000, 130, 2047, 64, 700], 64, 7
    Xs, *_ = _problems(sizes, d, 40)
    off = _offsets(Xs)
    X = np.concatenate(Xs)
    perm, tree = K.krr_cluster_batched(ctx, torch.from_numpy(X).cuda(), off, leaf, seed)
    perm = perm.cpu().numpy()
    for p, Xp in enumerate(Xs):
        lo, hi = off[p], off[p + 1]
        perm_o, tree_o, _ = cluster.two_means_tree(Xp, leaf, seed)
        assert np.array_equal(perm[lo:hi] - lo, perm_o), p
        a = tree_o.arrays()
        ref = {(int(b), int(e), bool(l < 0)) for b, e, l in zip(a["begin"], a["end"], a["left"])}
        assert _intervals(tree, lo, hi) == ref, p
    # the top joins the problems: the root covers everything
    root = len(tree["begin"]) - 1
    assert tree["begin"][root] == 0 and tree["end"][root] == len(X)


def _fit_batched(K, ctx, Xs, Ys, hs, lam, prec, eps_c, leaf, tol, **kw):
    off = _offsets(Xs)
    X = torch.from_numpy(np.concatenate(Xs)).cuda()
    Y = torch.from_numpy(np.ascontiguousarray(np.concatenate(Ys))).cuda()
    o = K.default_options(lambda_=lam, eps_c=eps_c, leaf=leaf, precision=prec, **kw)
    H = K.hss_compress_batched(ctx, X, off, hs, o)
    H.factor()
    a, res = H.solve(Y, tol=tol, max_refine=300)
    return H, a.cpu().numpy(), res, off


def test_batched_fp64_near_exact_matches_dense(K, ctx):
    """Three data sets, each at two widths (six problems); FP64 at a
    tolerance near round-off: one ULV solve gives each problem's dense
    solution."""
    Xd, yd, *_ = _problems([450, 1200, 257], 6, 50)
    Xs, Ys, hs = [], [], []
    for X, y in zip(Xd, yd):
        for h in (0.8, 1.5):
            Xs.append(X)
            Ys.append(y[:, None])
            hs.append(h)
    H, A, _, off = _fit_batched(K, ctx, Xs, Ys, hs, 1.0, K.KRR_FP64, 1e-13, 40, 0.0)
    for p, (X, y, h) in enumerate(zip(Xs, Ys, hs)):
        wd = solve.krr_dense(X.astype(np.float64), y[:, 0], h, 1.0)
        a = A[off[p]:off[p + 1], 0]
        assert np.linalg.norm(a - wd) <= 1e-8 * np.linalg.norm(wd), p
    H.close()


def test_batched_mixed_gmres_residual_and_prediction(K, ctx):
    """Eight problems, n in [512, 4096], d = 32, 16 right-hand sides, two
    widths; mixed precision, GMRES to 1e-5 over the batch.  Per problem the
    relative residual (oracle, FP64) is bounded by the batch tolerance times
    ||y_c|| / ||y_c restricted to the problem||; decision values match the
    oracle's product with the same weights."""
    rng = np.random.default_rng(9)
    sizes = [int(v) for v in rng.integers(512, 4097, size=4)]
    Xd, yd, Xtd, ytd = _problems(sizes, 32, 60, m_test=100)
    Xs, Ys, Xts, hs = [], [], [], []
    for k, (X, y, Xt) in enumerate(zip(Xd, yd, Xtd)):
        for h in (2.0, 4.0):
            Xs.append(X)
            Ys.append(np.concatenate([y[:, None], rng.standard_normal((len(y), 15))], 1))
            Xts.append(Xt)
            hs.append(h)
    tol = 1e-5
    H, A, res, off = _fit_batched(K, ctx, Xs, Ys, hs, 1.0, K.KRR_MIXED, 0.05, 128, tol)
    assert res <= tol
    Yall = np.concatenate(Ys)
    ynorm = np.linalg.norm(Yall, axis=0)
    for p, (X, Y, h) in enumerate(zip(Xs, Ys, hs)):
        a = A[off[p]:off[p + 1]]
        rho = solve.residual(X.astype(np.float64), h, 1.0, a, Y)
        bound = 2 * tol * ynorm / np.linalg.norm(Y, axis=0)
        assert np.all(rho <= bound), (p, rho.max())
    toff = _offsets(Xts)
    dec = H.predict(torch.from_numpy(np.concatenate(Xts)).cuda(), torch.from_numpy(A[:, :1].copy()).cuda(),
                    toff).cpu().numpy()[:, 0]
    for p, (X, Xt, h) in enumerate(zip(Xs, Xts, hs)):
        ref, ref_abs = kernel.kernel_product(Xt, X, h, A[off[p]:off[p + 1], :1], want_abs=True)
        err = np.abs(dec[toff[p]:toff[p + 1]] - ref[:, 0])
        assert np.all(err <= 1e-5 * ref_abs[:, 0] + 1e-9), p
    H.close()


def test_batched_equals_separate_handles(K, ctx):
    """FP64 at eps_c 1e-10 (both forms near exact): the batched handle's
    weights equal those of one handle per problem."""
    Xs, ys, *_ = _problems([600, 333, 900], 5, 70)
    hs = [1.0, 0.7, 1.3]
    H, A, _, off = _fit_batched(K, ctx, Xs, [y[:, None] for y in ys], hs, 0.5, K.KRR_FP64, 1e-10, 50, 0.0)
    H.close()
    for p, (X, y, h) in enumerate(zip(Xs, ys, hs)):
        o = K.default_options(h=h, lambda_=0.5, eps_c=1e-10, leaf=50, precision=K.KRR_FP64)
        Hp = K.hss_compress(ctx, torch.from_numpy(X).cuda(), o)
        Hp.factor()
        ap, _ = Hp.solve(torch.from_numpy(y[:, None].copy()).cuda())
        Hp.close()
        np.testing.assert_allclose(A[off[p]:off[p + 1], 0], ap.cpu().numpy()[:, 0], rtol=1e-7, atol=1e-10)


def test_batched_argument_errors(K, ctx):
    Xs, ys, *_ = _problems([200, 300], 4, 80)
    X = torch.from_numpy(np.concatenate(Xs)).cuda()
    o = K.default_options(lambda_=1.0, leaf=64, precision=K.KRR_FP64)
    for off, hs in [([0, 200, 400], [1.0, 1.0]),      # offsets do not end at n
                    ([0, 0, 500], [1.0, 1.0]),        # empty problem
                    ([0, 200, 500], [1.0, 0.0])]:     # width 0
        with pytest.raises(K.KRRError) as e:
            K.hss_compress_batched(ctx, X, off, hs, o)
        assert e.value.code == 1
    H = K.hss_compress_batched(ctx, X, [0, 200, 500], [1.0, 2.0], o)
    a = torch.zeros(500, 1, dtype=torch.float64, device="cuda")
    with pytest.raises(K.KRRError):
        H.predict(X[:10], a, [0, 5, 9])                # test offsets do not end at m
    with pytest.raises(K.KRRError):
        K.HSS.predict(H, X[:10], a)                    # the single-problem call refuses a batched handle
    H.close()


@pytest.mark.parametrize("d,h,eps_c", [(8, 4.0, 0.02), (32, 4.0, 0.05)])
def test_smooth_group_converges_with_fp64_factorization(K, ctx, d, h, eps_c):
    """Smooth kernels (d / h^2 <= 2 on standardized data: blocks large next
    to lambda = 1), which stall in GMRES behind an FP32 factorization: with
    the decompositions and factorization in FP64 (KRR_MIXED_F64, products
    still on tensor cores) a batch of such problems (n >= 4096 in all)
    reaches the tolerance, and every problem's residual against the FP64
    oracle's operator meets the bound."""
    sizes = [1500, 2048, 1111]
    Xs, ys, _, _ = _problems(sizes, d, 70 + d)
    off = _offsets(Xs)
    rng = np.random.default_rng(7)
    Ys = [np.concatenate([y[:, None], rng.standard_normal((len(y), 3))], 1) for y in ys]
    o = K.default_options(lambda_=1.0, eps_c=eps_c, eps_abs=1e-2, r_max=1024, leaf=128, seed=5,
                          flags=K.KRR_TRUNCATE_AT_RMAX | K.KRR_LAMBDA_TOL, precision=K.KRR_MIXED_F64)
    H = K.hss_compress_batched(ctx, torch.from_numpy(np.concatenate(Xs)).cuda(), off, [h] * len(sizes), o)
    H.factor()
    tol = 1e-4
    a, res = H.solve(torch.from_numpy(np.ascontiguousarray(np.concatenate(Ys))).cuda(), tol=tol, max_refine=600)
    assert 0 <= res <= tol
    A = a.cpu().numpy()
    for p in range(len(sizes)):
        rho = solve.residual(Xs[p].astype(np.float64), h, 1.0, A[off[p]:off[p + 1]], Ys[p])
        assert rho.max() <= 2 * tol, (p, rho)
    H.close()
