"""krr_standardize (Section 5.2: every feature to zero mean and unit
standard deviation; test points with the training statistics) against
the FP64 oracle, through the C-ABI, element by element.

The library accumulates the statistics in FP64 and rounds (x - mean) / std
once to FP32, so each output is within one FP32 ulp of the oracle's value
rounded to FP32 (the two FP64 sums differ only in summation order)."""
import numpy as np
import pytest
import torch

import synth
from oracle import prep

pytestmark = pytest.mark.gpu


def _within_ulp(got, want64):
    w32 = want64.astype(np.float32)
    ulp = np.spacing(np.abs(w32)).astype(np.float64)
    return np.abs(got.astype(np.float64) - want64) <= ulp + 1e-12


@pytest.mark.parametrize("n,m,d", [(65536, 4096, 8), (1000, 0, 54), (1, 3, 5)])
def test_standardize_matches_oracle(n, m, d):
    import paper_1803_10274_gb300 as K
    X, _, Xt, *_ = synth.mixture(n, d, 16, 0.7, 2, max(m, 1))
    X = (3.0 * X + 1.5).astype(np.float32)
    X[:, min(3, d - 1)] = 2.5                 # a column with zero spread: divided by 1
    Xt = (3.0 * Xt[:m] + 1.5).astype(np.float32)
    Z, Zt, mean, std = prep.standardize(X.astype(np.float64), Xt.astype(np.float64) if m else None)
    ctx = K.Context()
    try:
        Xd = torch.from_numpy(X).cuda()
        Xtd = torch.from_numpy(Xt).cuda() if m else None
        mu = torch.empty(d, dtype=torch.float64, device="cuda")
        sd = torch.empty(d, dtype=torch.float64, device="cuda")
        K.krr_standardize(ctx, Xd, Xtd, mu, sd)
        ctx.sync()
        np.testing.assert_allclose(mu.cpu().numpy(), mean, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(sd.cpu().numpy(), std, rtol=1e-12, atol=0)
        assert np.all(_within_ulp(Xd.cpu().numpy(), Z))
        if m:
            assert np.all(_within_ulp(Xtd.cpu().numpy(), Zt))
        assert np.all(Xd.cpu().numpy()[:, min(3, d - 1)] == 0.0)
    finally:
        ctx.close()
