"""Failure detection without a GPU fault: the pipelined tensor-core product
bounds every hand-off wait between its warps (TMA producer, MMA issuer,
epilogue).  With the limit set to one SM clock cycle, the first wait that
does not succeed at once runs out (the epilogue's first wait needs a TMA
load and a tensor-core GEMM, which take microseconds); the kernel then
stops its pipeline, lets the copies and MMAs it already issued finish,
frees its tensor memory and returns, and the context reports
KRR_ERR_TIMEOUT at the next synchronizing call.  The same context then
runs the product again with the default limit, and the result matches the
FP64 oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import kernel

pytestmark = pytest.mark.gpu

KRR_ERR_TIMEOUT = 6


def test_wait_limit_reports_timeout_and_context_recovers():
    import paper_1803_10274_gb300 as K
    n, d, r, h = 1024, 8, 64, 1.0
    X = synth.mixture(n, d, 4, 0.7, 41)[0].astype(np.float32)
    R = synth.gaussian_block(n, r, 42).astype(np.float32)
    Xd, Rd = torch.from_numpy(X).cuda(), torch.from_numpy(R).cuda()
    ctx = K.Context()
    try:
        ctx.set_wait_limit(1)
        S = K.krr_sample(ctx, Xd, Xd, h, 0.0, Rd)
        with pytest.raises(K.KRRError) as e:
            ctx.sync()
        assert e.value.code == KRR_ERR_TIMEOUT
        ctx.sync()                         # the latched status was cleared
        ctx.set_wait_limit(0)              # back to the default limit
        S = K.krr_sample(ctx, Xd, Xd, h, 0.0, Rd, S=S)
        ctx.sync()
        ref, ref_abs = kernel.kernel_product(X, X, h, R, want_abs=True)
        tol = 6e-4 * ref_abs + 3e-8 * np.abs(R).sum(0)[None, :] + 1e-6
        assert np.all(np.abs(S.cpu().numpy() - ref) <= tol)
    finally:
        ctx.close()
