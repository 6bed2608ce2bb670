"""Multi-class prediction by one-vs-all (Section 2 after Algorithm 1),
through the C-ABI: the c right-hand sides equal the oracle's bit for bit;
the argmax over the GPU's own decision values equals the oracle's argmax
rule applied to them (signed and literal |.| readings); accuracy is within
0.5 points of the oracle's dense FP64 multi-class solve."""
import numpy as np
import pytest
import torch

import synth
from oracle import prep, solve

pytestmark = pytest.mark.gpu


def test_one_vs_all_four_classes():
    import paper_1803_10274_gb300 as K
    n, m, c, h, lam = 4096, 1000, 4, 1.0, 1.0
    X, _, Xt, _, comp, comp_t = synth.mixture(n, 8, c, 0.7, 61, m)
    Z, Zt, _, _ = prep.standardize(X, Xt)
    Z32, Zt32 = Z.astype(np.float32), Zt.astype(np.float32)
    ctx = K.Context()
    try:
        cls = torch.from_numpy(comp.astype(np.int32)).cuda()
        Y = K.krr_one_vs_all(ctx, cls, c)
        Yo = solve.one_vs_all_targets(comp, c)
        assert np.array_equal(Y.cpu().numpy(), Yo)
        o = K.default_options(h=h, lambda_=lam, eps_c=0.05, leaf=128, precision=K.KRR_MIXED, seed=5)
        H = K.hss_compress(ctx, torch.from_numpy(Z32).cuda(), o)
        H.factor()
        A, res = H.solve(Y, tol=1e-4, max_refine=400)
        lab, dec = H.predict_classes(torch.from_numpy(Zt32).cuda(), A)
        lab_abs, _ = H.predict_classes(torch.from_numpy(Zt32).cuda(), A, absolute=True)
        dec = dec.cpu().numpy()
        assert np.array_equal(lab.cpu().numpy(), solve.predict_classes(dec))
        assert np.array_equal(lab_abs.cpu().numpy(), solve.predict_classes(dec, absolute=True))
        Zo, Zto = Z32.astype(np.float64), Zt32.astype(np.float64)
        W = solve.krr_dense(Zo, Yo, h, lam)
        lab_d = solve.predict_classes(solve.predict(Zto, Zo, W, h))
        acc = solve.accuracy(lab.cpu().numpy(), comp_t)
        acc_d = solve.accuracy(lab_d, comp_t)
        assert abs(acc - acc_d) <= 0.005, (acc, acc_d)
        assert acc_d > 0.5                          # four classes: far above chance
        H.close()
    finally:
        ctx.close()
