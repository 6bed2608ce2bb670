"""The allocation-free sampling entry point (krr_sample_noalloc) against
the allocating one (krr_sample), through the C-ABI.

Some callers cannot allocate device memory when they call the library
(a CUDA graph being captured, a fixed memory budget); krr_sample_noalloc
serves them from a fixed scratch array inside the library.  Both entry
points compute the same mixed-precision product, so each must agree with
the other within twice the bound the sampling tests use against the FP64
oracle.  Two calls in a row with different shapes check that the shared
scratch carries nothing from one call into the next.  This file is
collected last so that a failure here comes after every other test."""
import numpy as np
import pytest
import torch

import synth
from oracle import kernel

pytestmark = pytest.mark.gpu


def _bound(Sabs, R):
    return 2.0 * (6e-4 * Sabs + 3e-8 * np.abs(R).sum(0)[None, :] + 1e-6)


def test_noalloc_matches_allocating_entry_point():
    import paper_1803_10274_gb300 as K
    ctx = K.Context()
    try:
        # call 1: plain product, ragged sizes
        Xa = synth.mixture(3001, 8, 4, 0.7, 31)[0].astype(np.float32)
        Xb = synth.mixture(2500, 8, 4, 0.7, 32)[0].astype(np.float32)
        R = synth.gaussian_block(2500, 100, 33).astype(np.float32)
        Xad, Xbd, Rd = (torch.from_numpy(a).cuda() for a in (Xa, Xb, R))
        ref = K.krr_sample(ctx, Xad, Xbd, 1.2, 0.0, Rd)
        S1 = torch.full((3001, 100), float("nan"), device="cuda")
        K.krr_sample_noalloc(ctx, Xad, Xbd, 1.2, 0.0, Rd, S1)
        ctx.sync()
        _, Sabs = kernel.kernel_product(Xa, Xb, 1.2, R, want_abs=True)
        assert np.all(np.abs(S1.cpu().numpy() - ref.cpu().numpy()) <= _bound(Sabs, R))

        # call 2 right after: a different shape, same-leaf mask and lambda
        X = synth.mixture(1700, 6, 5, 0.7, 34)[0].astype(np.float32)
        R2 = synth.gaussian_block(1700, 64, 35).astype(np.float32)
        leaf = (np.arange(1700) * 5 // 77).astype(np.int32)
        Xd, R2d, Ld = (torch.from_numpy(a).cuda() for a in (X, R2, leaf))
        ref2 = K.krr_sample(ctx, Xd, Xd, 0.9, 2.0, R2d, Ld, Ld)
        S2 = torch.full((1700, 64), float("nan"), device="cuda")
        K.krr_sample_noalloc(ctx, Xd, Xd, 0.9, 2.0, R2d, S2, Ld, Ld)
        ctx.sync()
        _, Sabs2 = kernel.kernel_product(X, X, 0.9, R2, leaf, leaf, want_abs=True)
        assert np.all(np.abs(S2.cpu().numpy() - ref2.cpu().numpy()) <= _bound(Sabs2, R2))

        # beyond the fixed scratch: rejected before any GPU work
        big = torch.zeros(16385, 8, device="cuda")
        Rb = torch.zeros(16385, 8, device="cuda")
        Sb = torch.zeros(16385, 8, device="cuda")
        with pytest.raises(K.KRRError) as e:
            K.krr_sample_noalloc(ctx, big, big, 1.0, 0.0, Rb, Sb)
        assert e.value.code == 1
    finally:
        ctx.close()
