"""The allocation-free sampling entry point (krr_sample_noalloc), through
the C-ABI.

Some callers cannot allocate device memory at the moment they call the
library: a process that runs under a fixed device-memory budget, one that
has no allocator to hand to the library, or a latency-critical loop that
must not enter an allocator.  krr_sample_noalloc serves them from one
fixed scratch array inside the library.

Checked here, on two calls in a row with different shapes (so the shared
scratch must carry nothing from one call into the next):
* each result against the FP64 oracle, at the per-entry bound the sampling
  tests use for krr_sample, and against krr_sample itself;
* no allocation event in the context's allocator (torch's caching
  allocator) during a call;
* sizes beyond the fixed scratch are rejected with KRR_ERR_INVALID_ARG.
This file is collected last so that a failure here comes after every
other test."""
import numpy as np
import pytest
import torch

import synth
from oracle import kernel

pytestmark = pytest.mark.gpu


def _bound(Sabs, R):
    # the bound of the sampling tests: FP16 rounding of K, FP16 subnormals,
    # FP32 accumulation
    return 6e-4 * Sabs + 3e-8 * np.abs(R).sum(0)[None, :] + 1e-6


def _allocations():
    return torch.cuda.memory_stats().get("allocation.all.allocated", 0)


def test_noalloc_matches_oracle_and_allocates_nothing():
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
        torch.cuda.synchronize()
        a0 = _allocations()
        K.krr_sample_noalloc(ctx, Xad, Xbd, 1.2, 0.0, Rd, S1)
        ctx.sync()
        assert _allocations() == a0, "krr_sample_noalloc allocated device memory"
        S_exact, Sabs = kernel.kernel_product(Xa, Xb, 1.2, R, want_abs=True)
        tol = _bound(Sabs, R)
        got = S1.cpu().numpy()
        assert np.all(np.abs(got - S_exact) <= tol), float((np.abs(got - S_exact) / tol).max())
        assert np.all(np.abs(got - ref.cpu().numpy()) <= 2 * tol)

        # call 2 right after: another shape, d and h, same-leaf mask and lambda
        X = synth.mixture(1700, 6, 5, 0.7, 34)[0].astype(np.float32)
        R2 = synth.gaussian_block(1700, 64, 35).astype(np.float32)
        leaf = (np.arange(1700) * 5 // 77).astype(np.int32)
        Xd, R2d, Ld = (torch.from_numpy(a).cuda() for a in (X, R2, leaf))
        ref2 = K.krr_sample(ctx, Xd, Xd, 0.9, 2.0, R2d, Ld, Ld)
        S2 = torch.full((1700, 64), float("nan"), device="cuda")
        torch.cuda.synchronize()
        a0 = _allocations()
        K.krr_sample_noalloc(ctx, Xd, Xd, 0.9, 2.0, R2d, S2, Ld, Ld)
        ctx.sync()
        assert _allocations() == a0, "krr_sample_noalloc allocated device memory"
        S2_exact, Sabs2 = kernel.kernel_product(X, X, 0.9, R2, leaf, leaf, want_abs=True)
        S2_exact += 2.0 * R2.astype(np.float64)   # lambda R (R is FP16-exact)
        tol2 = _bound(Sabs2, R2)
        got2 = S2.cpu().numpy()
        assert np.all(np.abs(got2 - S2_exact) <= tol2), float((np.abs(got2 - S2_exact) / tol2).max())
        assert np.all(np.abs(got2 - ref2.cpu().numpy()) <= 2 * tol2)

        # beyond the fixed scratch: rejected before any GPU work
        big = torch.zeros(16385, 8, device="cuda")
        Rb = torch.zeros(16385, 8, device="cuda")
        Sb = torch.zeros(16385, 8, device="cuda")
        with pytest.raises(K.KRRError) as e:
            K.krr_sample_noalloc(ctx, big, big, 1.0, 0.0, Rb, Sb)
        assert e.value.code == 1
        wide = torch.zeros(64, 20, device="cuda")      # d = 20: 3d + 6 > 64
        Rw = torch.zeros(64, 8, device="cuda")
        Sw = torch.zeros(64, 8, device="cuda")
        with pytest.raises(K.KRRError) as e:
            K.krr_sample_noalloc(ctx, wide, wide, 1.0, 0.0, Rw, Sw)
        assert e.value.code == 1
    finally:
        ctx.close()
