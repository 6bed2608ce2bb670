"""The binding's argument rules for the fused-product entry points
(krr_sample, krr_sample_noalloc, krr_sample_f64).  The C calls see only
pointers, sizes and row strides, so every shape, dtype and layout mistake
must be caught before the call; each rule is exercised here on host
tensors (no GPU needed)."""
import pytest
import torch

from paper_1803_10274_gb300.binding import check_sample_args


def _ok(ma=5, nb=7, d=3, r=4, dt=torch.float32, leaves=False):
    Xa = torch.zeros(ma, d, dtype=dt)
    Xb = torch.zeros(nb, d, dtype=dt)
    R = torch.zeros(nb, r, dtype=dt)
    S = torch.zeros(ma, r, dtype=dt)
    la = torch.zeros(ma, dtype=torch.int32) if leaves else None
    lb = torch.zeros(nb, dtype=torch.int32) if leaves else None
    return dict(Xa=Xa, Xb=Xb, R=R, S=S, leaf_a=la, leaf_b=lb)


def _check(a, dt=torch.float32):
    check_sample_args(a["Xa"], a["Xb"], a["R"], a["S"], a["leaf_a"], a["leaf_b"], dt, cuda=False)


def test_valid_arguments_pass():
    _check(_ok())
    _check(_ok(leaves=True))
    _check(_ok(dt=torch.float64), torch.float64)
    a = _ok()
    a["S"] = torch.zeros(9, 6)             # a larger S is allowed
    _check(a)
    a = _ok()
    a["R"] = torch.zeros(7, 10)[:, :4]     # R with a row stride above r
    _check(a)


def test_xb_shape_must_match_r_rows_and_xa_columns():
    a = _ok()
    a["Xb"] = torch.zeros(6, 3)            # fewer rows than R
    with pytest.raises(ValueError, match="Xb"):
        _check(a)
    a = _ok()
    a["Xb"] = torch.zeros(7, 4)            # other feature count
    with pytest.raises(ValueError, match="Xb"):
        _check(a)


def test_s_must_hold_the_output():
    a = _ok()
    a["S"] = torch.zeros(4, 4)             # fewer rows than Xa
    with pytest.raises(ValueError, match="S must hold"):
        _check(a)
    a = _ok()
    a["S"] = torch.zeros(5, 3)             # fewer columns than R
    with pytest.raises(ValueError, match="S must hold"):
        _check(a)


def test_feature_rows_must_be_packed():
    a = _ok()
    a["Xa"] = torch.zeros(5, 8)[:, :3]     # column slice: row stride 8, not d
    with pytest.raises(ValueError, match="packed"):
        _check(a)
    a = _ok()
    a["Xb"] = torch.zeros(3, 7).t()        # transposed view
    with pytest.raises(ValueError, match="packed"):
        _check(a)


def test_r_and_s_row_major():
    a = _ok()
    a["R"] = torch.zeros(4, 7).t()
    with pytest.raises(ValueError, match="row-major"):
        _check(a)


def test_dtypes():
    a = _ok()
    a["R"] = torch.zeros(7, 4, dtype=torch.float64)
    with pytest.raises(ValueError, match="R must be"):
        _check(a)
    with pytest.raises(ValueError, match="Xa must be"):
        _check(_ok(), torch.float64)


def test_leaf_arrays():
    a = _ok(leaves=True)
    a["leaf_b"] = None                     # one without the other
    with pytest.raises(ValueError, match="both leaf arrays"):
        _check(a)
    a = _ok(leaves=True)
    a["leaf_a"] = torch.zeros(4, dtype=torch.int32)    # wrong length
    with pytest.raises(ValueError, match="leaf_a"):
        _check(a)
    a = _ok(leaves=True)
    a["leaf_b"] = torch.zeros(7, dtype=torch.int64)    # wrong dtype
    with pytest.raises(ValueError, match="leaf_b"):
        _check(a)
    a = _ok(leaves=True)
    a["leaf_a"] = torch.zeros(10, dtype=torch.int32)[::2]  # strided
    with pytest.raises(ValueError, match="contiguous"):
        _check(a)


def test_device_checked_by_default():
    a = _ok()
    with pytest.raises(ValueError, match="CUDA"):
        check_sample_args(a["Xa"], a["Xb"], a["R"], a["S"], None, None, torch.float32)


# ------------------------------------------------ krr_gemm_f32_batched
from paper_1803_10274_gb300.binding import check_gemm_args  # noqa: E402


def test_gemm_shapes_and_transposes():
    A, B, C = torch.zeros(2, 5, 7), torch.zeros(2, 7, 3), torch.zeros(2, 5, 3)
    assert check_gemm_args(A, B, C, False, False, cuda=False) == (2, 5, 3, 7)
    assert check_gemm_args(A.transpose(1, 2).contiguous(), B, None, True, False, cuda=False) == (2, 5, 3, 7)
    assert check_gemm_args(A, B.transpose(1, 2).contiguous(), C, False, True, cuda=False) == (2, 5, 3, 7)


@pytest.mark.parametrize("A,B,C", [
    (torch.zeros(2, 5, 7), torch.zeros(2, 6, 3), None),                  # inner dimensions differ
    (torch.zeros(2, 5, 7), torch.zeros(3, 7, 3), None),                  # batches differ
    (torch.zeros(2, 5, 7), torch.zeros(2, 7, 3), torch.zeros(2, 5, 4)),  # wrong C
    (torch.zeros(2, 5, 7, dtype=torch.float64), torch.zeros(2, 7, 3), None),
    (torch.zeros(5, 7), torch.zeros(7, 3), None),                        # 2-D, not batched
    (torch.zeros(2, 7, 5).transpose(1, 2), torch.zeros(2, 7, 3), None),  # not contiguous
])
def test_gemm_rejections(A, B, C):
    with pytest.raises(ValueError):
        check_gemm_args(A, B, C, False, False, cuda=False)


def test_gemm_needs_cuda_tensors():
    with pytest.raises(ValueError):
        check_gemm_args(torch.zeros(1, 2, 2), torch.zeros(1, 2, 2), None, False, False, cuda=True)


def test_gemm_sizes_within_int32():
    """Sizes and the count of 128 x 128 output tiles must fit the C ABI's
    int32 (K = 0 keeps the operands empty)."""
    with pytest.raises(ValueError):   # 2^17 x 2^17 tiles
        check_gemm_args(torch.zeros(1, 1 << 24, 0), torch.zeros(1, 0, 1 << 24), None, False, False, cuda=False)
    with pytest.raises(ValueError):   # M above 2^31 - 1
        check_gemm_args(torch.zeros(1, 1 << 31, 0), torch.zeros(1, 0, 1), None, False, False, cuda=False)
    assert check_gemm_args(torch.zeros(3, 1 << 12, 0), torch.zeros(3, 0, 1 << 12), None, False, False,
                           cuda=False) == (3, 1 << 12, 1 << 12, 0)
