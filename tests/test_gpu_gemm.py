"""The grouped FP32 product behind the interpolative decompositions' and the
factorization's node products, through the C-ABI (krr_gemm_f32_batched):
the tensor-core path (tcgen05 kind::tf32, operands split into two TF32
parts, three products) and the CUDA-core path against an FP64 product of
the same FP32 inputs, element by element at the bound

    |C - C_ref| <= (2^-20 + K 2^-23) (|alpha| |A| |B| + |beta| |C_in|)

(the split leaves out A_lo B_lo, about 2^-22 |a||b| per term; FP32
accumulation over K terms), on ragged shapes that span several 128 x 128
tiles and 32-wide K chunks, every transpose, and batches."""
import numpy as np
import pytest
import torch

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


def _ref(A, B, C0, alpha, beta, ta, tb):
    A64, B64 = A.double(), B.double()
    opA = A64.transpose(1, 2) if ta else A64
    opB = B64.transpose(1, 2) if tb else B64
    ref = alpha * torch.bmm(opA, opB) + beta * C0.double()
    mag = abs(alpha) * torch.bmm(opA.abs(), opB.abs()) + abs(beta) * C0.double().abs()
    return ref, mag


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("batch,M,N,Kd,ta,tb,alpha,beta", [
    (3, 200, 130, 300, False, False, 1.0, 0.0),
    (2, 129, 257, 33, True, False, -1.0, 1.0),
    (4, 64, 70, 1000, False, True, 0.5, 0.0),
    (1, 300, 45, 77, True, True, 1.0, -0.5),
    (5, 128, 128, 2032, False, True, 1.0, 0.0),     # a level of Gram matrices S S^T
])
def test_batched_product_matches_fp64(K, ctx, path, batch, M, N, Kd, ta, tb, alpha, beta):
    g = torch.Generator().manual_seed(batch * 1000 + M + N + Kd)
    A = torch.randn((batch, Kd, M) if ta else (batch, M, Kd), generator=g)
    B = torch.randn((batch, N, Kd) if tb else (batch, Kd, N), generator=g)
    C0 = torch.randn(batch, M, N, generator=g)
    C = K.krr_gemm_f32_batched(ctx, A.cuda(), B.cuda(), C0.clone().cuda(), alpha, beta, ta, tb, path)
    ctx.sync()
    ref, mag = _ref(A, B, C0, alpha, beta, ta, tb)
    err = (C.cpu().double() - ref).abs()
    bound = (2.0 ** -20 + Kd * 2.0 ** -23) * mag
    assert torch.all(err <= bound), float((err / bound).max())


def test_zero_k_scales_c(K, ctx):
    """K = 0: C = beta C on both paths."""
    C0 = torch.randn(2, 140, 150)
    for path in (1, 2):
        C = K.krr_gemm_f32_batched(ctx, torch.zeros(2, 140, 0).cuda(), torch.zeros(2, 0, 150).cuda(),
                                   C0.clone().cuda(), 1.0, 0.25, False, False, path)
        ctx.sync()
        assert torch.equal(C.cpu(), C0 * 0.25)


def test_argument_errors(K, ctx):
    A = torch.zeros(1, 4, 4, device="cuda")
    with pytest.raises(K.KRRError):
        K.krr_gemm_f32_batched(ctx, A, A, path=3)
    with pytest.raises(ValueError):
        K.krr_gemm_f32_batched(ctx, A, torch.zeros(1, 5, 4, device="cuda"))
