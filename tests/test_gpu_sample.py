"""Parity of the fused kernel x block product (the HSS sampling step) with
the FP64 oracle, through the C-ABI.

Mixed path bound, per entry (i, c):
  |S - S_exact| <= 6e-4 * sum_j K_ij |R_jc| + 3e-8 * sum_j |R_jc| + 1e-6
The first term covers rounding K to FP16 (half an ulp is 2^-11 relative
for normal values) plus the exponent and ex2 errors (~1e-5 relative); the
second the absolute rounding of subnormal FP16 values (2^-25); the third
FP32 accumulation.  R is FP16-representable, so it enters exactly.
FP64 path: relative 1e-12 of the same sum.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import kernel, rng

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


def _mixed_tol(Sabs, R):
    return 6e-4 * Sabs + 3e-8 * np.abs(R).sum(0)[None, :] + 1e-6


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("ma,nb,d,r,h", [(1000, 1000, 8, 64, 1.0),      # the small plain workload
                                         (777, 1313, 8, 40, 1.3),       # ragged tiles, padded columns
                                         (300, 129, 3, 256, 0.7),       # one column past a tile
                                         (1500, 2000, 19, 100, 2.0),    # one 64-wide feature chunk, full
                                         (700, 900, 33, 300, 1.5),      # two chunks, 2 launches of columns
                                         (640, 1000, 54, 100, 2.0),     # three chunks, one row-tile buffer
                                         (300, 513, 80, 64, 3.0),       # four chunks
                                         (1000, 1300, 8, 20, 1.0),      # 32-column product (10 GMRES columns x 2)
                                         (900, 700, 19, 32, 1.5),       # 32 columns, one 64-wide chunk
                                         (500, 600, 54, 7, 2.0)])       # 32 columns, three chunks
def test_mixed_matches_oracle(K, ctx, ma, nb, d, r, h):
    Xa = synth.mixture(ma, d, 4, 0.7, 10 + d)[0].astype(np.float32)
    Xb = synth.mixture(nb, d, 4, 0.7, 20 + d)[0].astype(np.float32)
    R = synth.gaussian_block(nb, r, 5).astype(np.float32)
    S = K.krr_sample(ctx, _cuda(Xa), _cuda(Xb), h, 0.0, _cuda(R))
    ctx.sync()
    ref, ref_abs = kernel.kernel_product(Xa, Xb, h, R, want_abs=True)
    err = np.abs(S.cpu().numpy() - ref)
    tol = _mixed_tol(ref_abs, R)
    assert np.all(err <= tol), float((err / tol).max())


@pytest.mark.parametrize("r", [64, 20])
def test_mixed_masked_and_lambda(K, ctx, r):
    n, d, h, lam = 1200, 8, 1.0, 4.0
    X = synth.mixture(n, d, 6, 0.7, 3)[0].astype(np.float32)
    R = synth.gaussian_block(n, r, 6).astype(np.float32)
    leaf = (np.arange(n) * 7 // 97).astype(np.int32)      # uneven leaves, not tile aligned
    Xd, Rd, Ld = _cuda(X), _cuda(R), _cuda(leaf)
    S = K.krr_sample(ctx, Xd, Xd, h, 0.0, Rd, Ld, Ld)
    S2 = K.krr_sample(ctx, Xd, Xd, h, lam, Rd)
    ctx.sync()
    ref, ref_abs = kernel.kernel_product(X, X, h, R, leaf, leaf, want_abs=True)
    assert np.all(np.abs(S.cpu().numpy() - ref) <= _mixed_tol(ref_abs, R))
    ref2, ref2_abs = kernel.kernel_product(X, X, h, R, want_abs=True)
    ref2 = ref2 + lam * R
    assert np.all(np.abs(S2.cpu().numpy() - ref2) <= _mixed_tol(ref2_abs, R))


@pytest.mark.parametrize("n,d,r,masked", [(4096, 40, 128, True),    # two chunks, two stages
                                           (4096, 54, 64, True),     # three chunks, two row-tile buffers
                                           (4096, 54, 128, False),   # three chunks, one row-tile buffer
                                           (3000, 80, 64, True),     # four chunks
                                           (3000, 100, 64, False),   # five chunks: rows streamed
                                           (4096, 128, 128, True),   # seven chunks, streamed
                                           (1500, 200, 200, True)])  # ten chunks, two column launches
def test_mixed_wide_rows_many_tiles_per_cta(K, ctx, n, d, r, masked):
    """Every CTA walks several tiles, so the stage / distance-buffer rings
    wrap; wide feature rows leave room for only two stages."""
    X = synth.mixture(n, d, 7, 0.7, 30 + d)[0]
    X = ((X - X.mean(0)) / X.std(0)).astype(np.float32)
    R = synth.gaussian_block(n, r, 8).astype(np.float32)
    h = 3.0 * np.sqrt(d / 54.0)
    leaf = (np.arange(n) // 100).astype(np.int32) if masked else None
    S = K.krr_sample(ctx, _cuda(X), _cuda(X), h, 0.0, _cuda(R), *(2 * [_cuda(leaf)] if masked else []))
    ctx.sync()
    rows = np.concatenate([np.arange(0, 130), np.arange(n - 130, n),
                           np.random.default_rng(1).choice(n, 100, replace=False)])
    ref, ref_abs = kernel.kernel_product(X, X, h, R, leaf, leaf, rows=rows, want_abs=True)
    err = np.abs(S.cpu().numpy()[rows] - ref)
    assert np.all(err <= _mixed_tol(ref_abs, R))


def test_mixed_full_size_sampled_rows(K, ctx):
    """The 65536-point, 8-feature, 64-column product the benchmark times,
    checked on 192 sampled rows (first, last and random)."""
    n, d, r, h = 65536, 8, 64, 1.0
    X = synth.mixture(n, d, 16, 0.7, 2)[0]
    X = ((X - X.mean(0)) / X.std(0)).astype(np.float32)
    R = synth.gaussian_block(n, r, 7).astype(np.float32)
    S = K.krr_sample(ctx, _cuda(X), _cuda(X), h, 0.0, _cuda(R))
    ctx.sync()
    rows = np.concatenate([[0, 1, 127, 128, n - 1], np.random.default_rng(0).choice(n, 187, replace=False)])
    ref, ref_abs = kernel.kernel_product(X, X, h, R, rows=rows, want_abs=True)
    err = np.abs(S.cpu().numpy()[rows] - ref)
    assert np.all(err <= _mixed_tol(ref_abs, R))


def test_mixed_image_like_d784(K, ctx):
    """MNIST-shaped rows (d = 784, about 80 % exact zeros, values in [0, 1],
    h = 4): 37 streamed feature chunks, masked by leaves."""
    n, r, h = 2048, 64, 4.0
    X = synth.image_like(n, 3)[0].astype(np.float32)
    R = synth.gaussian_block(n, r, 9).astype(np.float32)
    leaf = (np.arange(n) // 200).astype(np.int32)
    S = K.krr_sample(ctx, _cuda(X), _cuda(X), h, 0.0, _cuda(R), _cuda(leaf), _cuda(leaf))
    ctx.sync()
    rows = np.concatenate([np.arange(0, 130), np.arange(n - 130, n)])
    ref, ref_abs = kernel.kernel_product(X, X, h, R, leaf, leaf, rows=rows, want_abs=True)
    err = np.abs(S.cpu().numpy()[rows] - ref)
    assert np.all(err <= _mixed_tol(ref_abs, R))


def test_mixed_one_million_points_sampled_rows(K, ctx):
    """n = 1,048,576, d = 8, r = 256 (the batched workload's single large
    product): 48 sampled rows against the oracle."""
    n, d, r = 1 << 20, 8, 256
    X = synth.mixture(n, d, 16, 0.7, 6)[0]
    X = ((X - X.mean(0)) / X.std(0)).astype(np.float32)
    R = synth.gaussian_block(n, r, 6).astype(np.float32)
    S = K.krr_sample(ctx, _cuda(X), _cuda(X), 1.0, 0.0, _cuda(R))
    ctx.sync()
    rows = np.concatenate([[0, 127, 128, n - 1], np.random.default_rng(2).choice(n, 44, replace=False)])
    ref, ref_abs = kernel.kernel_product(X, X, 1.0, R, rows=rows, want_abs=True)
    err = np.abs(S[torch.from_numpy(rows).cuda()].cpu().numpy() - ref)
    assert np.all(err <= _mixed_tol(ref_abs, R))


@pytest.mark.parametrize("ma,nb,d,r", [(500, 700, 8, 64), (129, 65, 54, 10)])
def test_f64_matches_oracle(K, ctx, ma, nb, d, r):
    Xa = synth.mixture(ma, d, 4, 0.7, 1)[0]
    Xb = synth.mixture(nb, d, 4, 0.7, 2)[0]
    R = np.random.default_rng(3).standard_normal((nb, r))
    la = (np.arange(ma) // 50).astype(np.int32)
    lb = (np.arange(nb) // 40).astype(np.int32)
    S = K.krr_sample_f64(ctx, _cuda(Xa), _cuda(Xb), 0.9, 0.0, _cuda(R), _cuda(la), _cuda(lb))
    ctx.sync()
    ref, ref_abs = kernel.kernel_product(Xa, Xb, 0.9, R, la, lb, want_abs=True)
    assert np.all(np.abs(S.cpu().numpy() - ref) <= 1e-12 * ref_abs + 1e-300)


def test_random_block_matches_oracle(K, ctx):
    n, r, col0, seed = 257, 12, 8, 99
    want = rng.gaussian_block(n, r, seed, col0=col0)
    got64 = K.krr_random_block(ctx, n, r, col0, seed, K.KRR_FP64).cpu().numpy()
    got16 = K.krr_random_block(ctx, n, r, col0, seed, K.KRR_MIXED).cpu().numpy()
    ctx.sync()
    np.testing.assert_allclose(got64, want, rtol=1e-13, atol=1e-13)
    w16 = want.astype(np.float16).astype(np.float64)
    diff = np.abs(got16 - w16)
    ulp = np.abs(np.spacing(w16.astype(np.float16))).astype(np.float64)
    assert np.all(diff <= ulp)                      # equal except a rare rounding tie
    assert np.mean(diff == 0) > 0.999


@pytest.mark.parametrize("ma,nb,d,r,masked", [(3000, 2500, 8, 64, False), (2048, 2048, 8, 256, True),
                                              (1500, 1500, 30, 100, False)])
def test_autotuned_product_matches_oracle(K, ma, nb, d, r, masked):
    """With the autotuner on, the first call of a shape class times every
    launch variant on the call itself (clearing S before each trial) and
    leaves the fastest one's result; the second call uses the cached
    choice.  Both match the oracle at the mixed bound."""
    c = K.Context()
    try:
        c.set_autotune(True)
        Xa = synth.mixture(ma, d, 4, 0.7, 60 + d)[0].astype(np.float32)
        Xb = synth.mixture(nb, d, 4, 0.7, 61 + d)[0].astype(np.float32) if not masked else Xa
        R = synth.gaussian_block(Xb.shape[0], r, 62).astype(np.float32)
        leaf = (np.arange(Xa.shape[0]) // 128).astype(np.int32) if masked else None
        args = [_cuda(leaf), _cuda(leaf)] if masked else []
        ref, ref_abs = kernel.kernel_product(Xa, Xb, 1.1, R, leaf, leaf, want_abs=True)
        for _ in range(2):
            S = K.krr_sample(c, _cuda(Xa), _cuda(Xb), 1.1, 0.0, _cuda(R), *args)
            c.sync()
            assert np.all(np.abs(S.cpu().numpy() - ref) <= _mixed_tol(ref_abs, R))
    finally:
        c.close()
