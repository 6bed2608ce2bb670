"""GPU parity of the held-out loss gradient (krr_heldout_grad and the
autograd Function above it) against the oracle's dense FP64 gradient and
central finite differences (step 1e-4)."""
import numpy as np
import pytest
import torch

import synth
from oracle import grad, prep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kx():
    import paper_1803_10274_gb300 as k
    return k, k.Context()


def _data(n, m, d, n_comp, seed, cls=None):
    X, y, Xt, yt, c, ct = synth.mixture(n, d, n_comp, 0.7, seed, m)
    if cls is not None:
        y, yt = synth.labels_one_vs_rest(c, cls), synth.labels_one_vs_rest(ct, cls)
    Z, Zt, _, _ = prep.standardize(X, Xt)
    return Z.astype(np.float32), Zt.astype(np.float32), y, yt


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _gpu_grad(k, ctx, X, Xt, y, yt, h, lam, prec, eps_c, leaf, tol, grad_=True):
    o = k.default_options(h=h, lambda_=lam, eps_c=eps_c, leaf=leaf, precision=prec)
    H = k.hss_compress(ctx, _dev(X, torch.float32), o)
    try:
        return H.heldout_grad(_dev(Xt, torch.float32), _dev(y, torch.float64), _dev(yt, torch.float64), tol=tol,
                              max_refine=300, grad=grad_, want_alpha=True)
    finally:
        H.close()


def test_grad_fp64_matches_dense_oracle(kx):
    k, ctx = kx
    X, Xt, y, yt = _data(700, 180, 6, 4, 11)
    h, lam = 1.2, 0.8
    r = _gpu_grad(k, ctx, X, Xt, y, yt, h, lam, k.KRR_FP64, 1e-10, 64, 1e-12)
    L, dh, dl, dX = grad.loss_and_grad(X.astype(np.float64), Xt.astype(np.float64), y, yt, h, lam)
    assert abs(r["loss"] - L) <= 1e-9 * L
    assert abs(r["dh"] - dh) <= 1e-8 * abs(dh)
    assert abs(r["dlambda"] - dl) <= 1e-8 * abs(dl)
    gX = r["dX"].cpu().numpy()
    assert np.abs(gX - dX).max() <= 1e-8 * np.abs(dX).max()


def test_grad_fp64_matches_central_differences(kx):
    """The GPU loss itself, differenced with step 1e-4, against the GPU
    adjoint gradient (FP64 solves to 1e-12, so the difference quotient is
    limited by its O(step^2) truncation)."""
    k, ctx = kx
    X, Xt, y, yt = _data(500, 120, 5, 4, 12)
    h, lam, st = 0.9, 0.6, 1e-4
    f = lambda X_, h_, l_: _gpu_grad(k, ctx, X_, Xt, y, yt, h_, l_, k.KRR_FP64, 1e-10, 64, 1e-12,
                                     grad_=False)["loss"]
    r = _gpu_grad(k, ctx, X, Xt, y, yt, h, lam, k.KRR_FP64, 1e-10, 64, 1e-12)
    fd_h = (f(X, h + st, lam) - f(X, h - st, lam)) / (2 * st)
    fd_l = (f(X, h, lam + st) - f(X, h, lam - st)) / (2 * st)
    assert abs(r["dh"] - fd_h) <= 1e-5 * max(1.0, abs(fd_h))
    assert abs(r["dlambda"] - fd_l) <= 1e-5 * max(1.0, abs(fd_l))
    gX = r["dX"].cpu().numpy()
    # X is FP32 on the device: perturb in FP64 by a representable step
    for p, q in [(3, 0), (250, 2), (499, 4)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[p, q] += np.float32(st)
        Xm[p, q] -= np.float32(st)
        fd = (f(Xp, h, lam) - f(Xm, h, lam)) / (float(Xp[p, q]) - float(Xm[p, q]))
        assert abs(gX[p, q] - fd) <= 1e-5 * max(1.0, np.abs(gX).max())


@pytest.mark.parametrize("n,m", [(4096, 1024), (3000, 700)])
def test_grad_mixed_d54_matches_dense_oracle(kx, n, m):
    """COVTYPE-shaped (d=54, 7 classes, one-vs-rest for class 2) mixed path
    vs the dense FP64 gradient.  The fused products split K and the columns
    into FP16 hi/lo pairs (about 2^-22 relative per term, FP32 accumulation),
    which puts the floor of the solves' relative residual near 3e-7; both
    solves stop at 1e-6.  Observed errors are near 3e-6 (loss, dh,
    dlambda) and 3e-5 of max |dX|; the bounds leave a factor of ten."""
    k, ctx = kx
    X, Xt, y, yt = _data(n, m, 54, 7, 4, cls=2)
    h, lam = 3.0, 1.0
    r = _gpu_grad(k, ctx, X, Xt, y, yt, h, lam, k.KRR_MIXED, 0.05, 128, 1e-6)
    L, dh, dl, dX = grad.loss_and_grad(X.astype(np.float64), Xt.astype(np.float64), y, yt, h, lam)
    assert abs(r["loss"] - L) <= 3e-5 * L
    assert abs(r["dh"] - dh) <= 3e-5 * abs(dh)
    assert abs(r["dlambda"] - dl) <= 1e-4 * abs(dl)
    gX = r["dX"].cpu().numpy()
    assert np.abs(gX - dX).max() <= 3e-4 * np.abs(dX).max()


def test_loss_only_matches_full_call(kx):
    """The loss-only call runs the same solve and held-out product.  The
    fused product adds row-tile partial sums atomically, so the two agree
    to FP32 rounding of the sums, not bit for bit."""
    k, ctx = kx
    X, Xt, y, yt = _data(1500, 300, 54, 7, 5, cls=2)
    a = _gpu_grad(k, ctx, X, Xt, y, yt, 3.0, 1.0, k.KRR_MIXED, 0.05, 128, 1e-6, grad_=False)
    b = _gpu_grad(k, ctx, X, Xt, y, yt, 3.0, 1.0, k.KRR_MIXED, 0.05, 128, 1e-6)
    assert "dX" not in a
    assert abs(a["loss"] - b["loss"]) <= 2e-6 * b["loss"]
    da = (a["alpha"] - b["alpha"]).abs().max().item()
    assert da <= 2e-6 * b["alpha"].abs().max().item()


def test_autograd_function_backward(kx):
    k, ctx = kx
    X, Xt, y, yt = _data(800, 200, 8, 4, 13)
    Xd = _dev(X, torch.float32).requires_grad_(True)
    h = torch.tensor(1.1, dtype=torch.float64, device="cuda", requires_grad=True)
    lam = torch.tensor(0.9, dtype=torch.float64, device="cuda", requires_grad=True)
    o = k.default_options(eps_c=1e-10, leaf=64, precision=k.KRR_FP64)
    L = k.krr_heldout_loss(ctx, Xd, h, lam, _dev(Xt, torch.float32), _dev(y, torch.float64),
                           _dev(yt, torch.float64), opts=o, tol=1e-12)
    (3.0 * L).backward()
    L0, dh, dl, dX = grad.loss_and_grad(X.astype(np.float64), Xt.astype(np.float64), y, yt, 1.1, 0.9)
    assert abs(L.item() - L0) <= 1e-9 * L0
    assert abs(h.grad.item() - 3 * dh) <= 1e-7 * abs(3 * dh)
    assert abs(lam.grad.item() - 3 * dl) <= 1e-7 * abs(3 * dl)
    assert Xd.grad.dtype == torch.float32
    assert np.abs(Xd.grad.cpu().numpy() - 3 * dX).max() <= 1e-6 * np.abs(3 * dX).max()


def test_grad_full_size_matches_dense_oracle(kx):
    """n=16384, d=54, 4096 held out: the size the gradient is timed at, on
    the mixed path, against the dense FP64 gradient (the oracle's dense
    matrices take about 10 GB of host memory and half a minute).  dX_p
    scales with alpha_p and z_p one by one, so its error follows their
    componentwise error: up to cond(K + lambda I) times the solves'
    relative residual (1e-6), with cond near 1 + ||K|| / lambda ~ 300 here
    (observed 5e-4 of max |dX|)."""
    k, ctx = kx
    X, Xt, y, yt = _data(16384, 4096, 54, 7, 4, cls=2)
    h, lam = 3.0, 1.0
    r = _gpu_grad(k, ctx, X, Xt, y, yt, h, lam, k.KRR_MIXED, 0.1, 128, 1e-6)
    L, dh, dl, dX = grad.loss_and_grad(X.astype(np.float64), Xt.astype(np.float64), y, yt, h, lam)
    assert abs(r["loss"] - L) <= 3e-5 * L
    assert abs(r["dh"] - dh) <= 1e-4 * abs(dh)
    assert abs(r["dlambda"] - dl) <= 1e-4 * abs(dl)
    gX = r["dX"].cpu().numpy()
    assert np.abs(gX - dX).max() <= 3e-3 * np.abs(dX).max()
    assert np.linalg.norm(gX - dX) <= 1e-3 * np.linalg.norm(dX)


def test_grad_bad_arguments(kx):
    k, ctx = kx
    X, Xt, y, yt = _data(300, 50, 4, 3, 14)
    o = k.default_options(h=1.0, lambda_=1.0, leaf=64, precision=k.KRR_FP64)
    H = k.hss_compress(ctx, _dev(X, torch.float32), o)
    try:
        with pytest.raises(k.KRRError) as e:
            H.heldout_grad(_dev(Xt[:0], torch.float32), _dev(y, torch.float64), _dev(yt[:0], torch.float64))
        assert e.value.code == 1
    finally:
        H.close()
