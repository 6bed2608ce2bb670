"""The compressed HSS matrix H itself, through the C-ABI (hss_matvec applies
H from its generators: leaf blocks, nested interpolative bases, sibling
blocks; Section 3.1).

* Compression error: ||H x - (K + lambda I) x|| / ||(K + lambda I) x|| is
  O(eps_c) against the FP64 oracle's exact product, at real (intermediate)
  ranks.
* ULV identity: the ULV factorization eliminates exactly H, so one ULV
  solve (no refinement) of H x returns x to rounding times the condition
  number: ||x' - x|| / ||x|| <= 100 u kappa(K + lambda I), with u the unit
  roundoff of the factorization (FP64, or FP32 in the mixed path) and
  kappa from the oracle's dense eigenvalues.  A wrong but nonsingular
  factorization fails this even though it would still precondition GMRES.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import kernel, prep

pytestmark = pytest.mark.gpu


def _kappa(X, h, lam):
    A = kernel.kernel_matrix(X, X, h)
    A[np.diag_indices_from(A)] += lam
    w = np.linalg.eigvalsh(A)
    return float(w[-1] / w[0])


@pytest.mark.parametrize("prec,eps_c,n,r0", [("fp64", 1e-4, 2048, 64), ("fp64", 1e-6, 2048, 64),
                                             ("mixed", 0.05, 2048, 64), ("mixed", 0.05, 8192, 64),
                                             ("fp64", 1e-4, 2048, 16), ("mixed", 0.05, 8192, 16)])
def test_hss_matvec_and_ulv_identity(prec, eps_c, n, r0):
    """r0 = 16: several adaptive rounds (every decomposition recomputed with
    the doubled sample count); the same gates hold."""
    import paper_1803_10274_gb300 as K
    h, lam, leaf = 1.0, 1.0, 64
    X = synth.mixture(n, 8, 8, 0.7, 51)[0]
    Z = prep.standardize(X)[0].astype(np.float32)
    Zo = Z.astype(np.float64)
    x = np.random.default_rng(52).standard_normal((n, 4))
    ctx = K.Context()
    try:
        P = K.KRR_FP64 if prec == "fp64" else K.KRR_MIXED
        o = K.default_options(h=h, lambda_=lam, eps_c=eps_c, leaf=leaf, precision=P, seed=3, r0=r0)
        H = K.hss_compress(ctx, torch.from_numpy(Z).cuda(), o)
        st = H.stats()
        assert 0 < st["max_rank"] < n // 2          # real ranks, neither 0 nor full
        if r0 == 16:
            assert st["rounds"] >= 3, st
        xd = torch.from_numpy(x).cuda()
        Hx = H.matvec(xd)
        Ax = kernel.kernel_product(Zo, Zo, h, x) + lam * x
        rel = np.linalg.norm(Hx.cpu().numpy() - Ax) / np.linalg.norm(Ax)
        assert rel <= 10 * eps_c, rel
        H.factor()
        xs, _ = H.solve(Hx, tol=0.0)
        err = np.linalg.norm(xs.cpu().numpy() - x) / np.linalg.norm(x)
        u = 2.0 ** -53 if prec == "fp64" else 2.0 ** -24
        kap = _kappa(Zo, h, lam) if n <= 4096 else _kappa(Zo[:4096], h, lam) * n / 4096
        assert err <= 100 * u * kap, (err, kap)
        H.close()
    finally:
        ctx.close()
