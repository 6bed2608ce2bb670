"""Functions with the names of the C entry points, taking torch tensors.

Argument marshalling only: shapes and dtypes are checked, pointers are
passed to the C library, errors become KRRError.
"""
from __future__ import annotations

import atexit
import ctypes
import weakref

import torch

from . import _lib
from ._lib import (KRR_FP64, KRR_LAMBDA_TOL, KRR_MIXED, KRR_MIXED_F64, KRR_ORDER_KD, KRR_ORDER_NATURAL, KRR_ORDER_PCA,
                   KRR_ORDER_TWO_MEANS, KRR_TRUNCATE_AT_RMAX, KRRError, check, lib)

__all__ = ["Context", "KRRError", "KRR_MIXED", "KRR_FP64", "KRR_MIXED_F64", "KRR_TRUNCATE_AT_RMAX", "KRR_LAMBDA_TOL", "KRR_ORDER_TWO_MEANS",
           "KRR_ORDER_NATURAL", "KRR_ORDER_KD", "KRR_ORDER_PCA", "krr_order", "krr_standardize", "krr_cluster", "krr_sample",
           "krr_sample_f64", "krr_sample_noalloc", "krr_random_block", "krr_one_vs_all", "krr_gemm_f32_batched", "krr_h_partition", "HSS", "hss_compress", "default_options",
           "HeldOutLoss", "krr_heldout_loss", "krr_cluster_batched", "hss_compress_batched", "lib"]


_shutting_down = [False]


@atexit.register
def _mark_shutdown():
    # Handles still open at interpreter exit are not destroyed: their
    # device memory goes back through callbacks into torch, which may
    # already be finalized.  The process is ending; the driver reclaims it.
    _shutting_down[0] = True


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, name, dims=2):
    if t is None:
        return
    if not (t.is_cuda and t.dtype == dtype and t.dim() == dims):
        raise ValueError("%s must be a %d-D CUDA %s tensor" % (name, dims, dtype))
    if dims == 2 and t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("%s must be row-major (unit column stride)" % name)


class Context:
    """A krr_ctx bound to torch's current stream and caching allocator."""

    def __init__(self, stream: torch.cuda.Stream | None = None, torch_allocator: bool = True):
        self.stream = stream or torch.cuda.current_stream()
        self.device = torch.cuda.current_device()
        self._keep = []
        self._handles = weakref.WeakSet()  # HSS handles made on this context
        al = None
        if torch_allocator:
            dev, st = self.device, self.stream

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:
                    return None

            def _free(p, user):
                torch.cuda.caching_allocator_delete(p)

            al = _lib.krr_allocator(_lib.krr_allocator._fields_[0][1](_alloc),
                                    _lib.krr_allocator._fields_[1][1](_free), None)
            self._keep.append(al)
        h = ctypes.c_void_p()
        check(lib().krr_create(ctypes.byref(h), ctypes.byref(al) if al else None,
                               ctypes.c_void_p(self.stream.cuda_stream)))
        self.h = h

    def sync(self):
        check(lib().krr_sync(self.h))

    def probe_rate(self, which):
        """krr_probe_rate: 0 FP32 FMA flop/s, 1 FP64 FMA flop/s, 2 ex2/s,
        3 FP32->FP16 conversions/s."""
        v = ctypes.c_double()
        check(lib().krr_probe_rate(self.h, int(which), ctypes.byref(v)))
        return v.value

    def set_autotune(self, enable=True):
        """Time the fused product's launch variants per shape class on first
        use and keep the fastest (krr_set_autotune)."""
        check(lib().krr_set_autotune(self.h, 1 if enable else 0))

    def set_wait_limit(self, cycles=0):
        """Limit of each device-side hand-off wait of the pipelined kernels
        launched from now on, in SM clock cycles (0: the default)."""
        check(lib().krr_set_wait_limit(self.h, int(cycles)))

    def close(self):
        if getattr(self, "h", None):
            # handles made on this context are freed through it: close them first
            for hss in list(getattr(self, "_handles", ())):
                hss.close()
            if not _shutting_down[0]:
                lib().krr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def krr_standardize(ctx, X, Xt=None, mean=None, std=None):
    _need(X, torch.float32, "X")
    _need(Xt, torch.float32, "Xt")
    n, d = X.shape
    m = 0 if Xt is None else Xt.shape[0]
    check(lib().krr_standardize(ctx.h, _ptr(X), n, d, _ptr(Xt), m, _ptr(mean), _ptr(std)))


def krr_cluster(ctx, X, leaf, seed):
    """Returns (perm (device int32), tree dict of host int32 numpy arrays)."""
    import numpy as np
    _need(X, torch.float32, "X")
    n, d = X.shape
    perm = torch.empty(n, dtype=torch.int32, device=X.device)
    cap = max(2 * n, 1)
    arrs = {k: np.zeros(cap, np.int32) for k in ("begin", "end", "left", "right", "parent", "level")}
    ta = _lib.krr_tree_arrays(**{k: v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for k, v in arrs.items()})
    nn = ctypes.c_int32()
    check(lib().krr_cluster(ctx.h, _ptr(X), n, d, leaf, seed, _ptr(perm), cap, ta, ctypes.byref(nn)))
    return perm, {k: v[:nn.value].copy() for k, v in arrs.items()}


def krr_order(ctx, X, leaf, ordering, seed=1):
    """Ordering of Section 4.3 (KRR_ORDER_*): (perm, tree dict) as krr_cluster."""
    import numpy as np
    _need(X, torch.float32, "X")
    n, d = X.shape
    perm = torch.empty(n, dtype=torch.int32, device=X.device)
    cap = max(2 * n, 1)
    arrs = {k: np.zeros(cap, np.int32) for k in ("begin", "end", "left", "right", "parent", "level")}
    ta = _lib.krr_tree_arrays(**{k: v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for k, v in arrs.items()})
    nn = ctypes.c_int32()
    check(lib().krr_order(ctx.h, _ptr(X), n, d, leaf, ordering, seed, _ptr(perm), cap, ta, ctypes.byref(nn)))
    return perm, {k: v[:nn.value].copy() for k, v in arrs.items()}


def _i64_array(v):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int64))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def krr_cluster_batched(ctx, X, offsets, leaf, seed):
    """Two-means order of many problems at once (rows split by offsets)."""
    import numpy as np
    _need(X, torch.float32, "X")
    n, d = X.shape
    off, offp = _i64_array(offsets)
    perm = torch.empty(n, dtype=torch.int32, device=X.device)
    cap = max(2 * n, 1)
    arrs = {k: np.zeros(cap, np.int32) for k in ("begin", "end", "left", "right", "parent", "level")}
    ta = _lib.krr_tree_arrays(**{k: v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for k, v in arrs.items()})
    nn = ctypes.c_int32()
    check(lib().krr_cluster_batched(ctx.h, _ptr(X), n, d, len(off) - 1, offp, leaf, seed, _ptr(perm), cap, ta,
                                    ctypes.byref(nn)))
    return perm, {k: v[:nn.value].copy() for k, v in arrs.items()}


def check_sample_args(Xa, Xb, R, S, leaf_a, leaf_b, dtype, cuda=True):
    """Shapes, dtypes and layouts the C entry points of the fused product
    rely on (they see only pointers, sizes and row strides): Xa (ma x d) and
    Xb (nb x d) packed row-major, R (nb x r) and S (at least ma x r)
    row-major, leaf arrays both given or both absent, int32 of length ma and
    nb.  Raises ValueError; with cuda=False the device is not checked (the
    rules themselves are tested on the host)."""
    for t, name in ((Xa, "Xa"), (Xb, "Xb"), (R, "R"), (S, "S")):
        if not torch.is_tensor(t) or t.dtype != dtype or t.dim() != 2:
            raise ValueError("%s must be a 2-D %s tensor" % (name, dtype))
        if cuda and not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
    ma, d = Xa.shape
    nb, r = R.shape
    if d < 1 or r < 1:
        raise ValueError("d and r must be positive")
    if tuple(Xb.shape) != (nb, d):
        raise ValueError("Xb must be %d x %d (rows of R x columns of Xa), got %s" % (nb, d, tuple(Xb.shape)))
    for t, name in ((Xa, "Xa"), (Xb, "Xb")):
        if t.shape[0] > 1 and t.stride(0) != d or d > 1 and t.stride(1) != 1:
            raise ValueError("%s must be packed row-major (row stride %d)" % (name, d))
    if S.shape[0] < ma or S.shape[1] < r:
        raise ValueError("S must hold at least %d x %d, got %s" % (ma, r, tuple(S.shape)))
    for t, name in ((R, "R"), (S, "S")):
        if t.shape[1] > 1 and t.stride(1) != 1:
            raise ValueError("%s must be row-major (unit column stride)" % name)
        if t.shape[0] > 1 and t.stride(0) < r:
            raise ValueError("%s row stride must be at least r = %d" % (name, r))
    if (leaf_a is None) != (leaf_b is None):
        raise ValueError("give both leaf arrays or neither")
    if leaf_a is not None:
        for t, name, ln in ((leaf_a, "leaf_a", ma), (leaf_b, "leaf_b", nb)):
            if not torch.is_tensor(t) or t.dtype != torch.int32 or t.dim() != 1 or t.shape[0] != ln:
                raise ValueError("%s must be a 1-D int32 tensor of length %d" % (name, ln))
            if ln > 1 and t.stride(0) != 1:
                raise ValueError("%s must be contiguous" % name)
            if cuda and not t.is_cuda:
                raise ValueError("%s must be a CUDA tensor" % name)


def krr_sample(ctx, Xa, Xb, h, lam, R, leaf_a=None, leaf_b=None, S=None):
    if S is None and torch.is_tensor(Xa) and torch.is_tensor(R) and Xa.dim() == 2 and R.dim() == 2:
        S = torch.empty(Xa.shape[0], R.shape[1], dtype=torch.float32, device=Xa.device)
    check_sample_args(Xa, Xb, R, S, leaf_a, leaf_b, torch.float32)
    ma, d = Xa.shape
    nb, r = R.shape
    check(lib().krr_sample(ctx.h, _ptr(Xa), ma, _ptr(Xb), nb, d, h, lam, _ptr(R), r, R.stride(0),
                           _ptr(leaf_a), _ptr(leaf_b), _ptr(S), S.stride(0)))
    return S


def krr_sample_noalloc(ctx, Xa, Xb, h, lam, R, S, leaf_a=None, leaf_b=None):
    """krr_sample into a caller-provided S, with no device allocation in
    the library (fixed internal scratch; see include/krrhss.h for limits)."""
    check_sample_args(Xa, Xb, R, S, leaf_a, leaf_b, torch.float32)
    ma, d = Xa.shape
    nb, r = R.shape
    check(lib().krr_sample_noalloc(ctx.h, _ptr(Xa), ma, _ptr(Xb), nb, d, h, lam, _ptr(R), r, R.stride(0),
                                   _ptr(leaf_a), _ptr(leaf_b), _ptr(S), S.stride(0)))
    return S


def krr_sample_f64(ctx, Xa, Xb, h, lam, R, leaf_a=None, leaf_b=None, S=None):
    if S is None and torch.is_tensor(Xa) and torch.is_tensor(R) and Xa.dim() == 2 and R.dim() == 2:
        S = torch.empty(Xa.shape[0], R.shape[1], dtype=torch.float64, device=Xa.device)
    check_sample_args(Xa, Xb, R, S, leaf_a, leaf_b, torch.float64)
    ma, d = Xa.shape
    nb, r = R.shape
    check(lib().krr_sample_f64(ctx.h, _ptr(Xa), ma, _ptr(Xb), nb, d, h, lam, _ptr(R), r, R.stride(0),
                               _ptr(leaf_a), _ptr(leaf_b), _ptr(S), S.stride(0)))
    return S


def krr_random_block(ctx, n, r, col0, seed, precision=KRR_MIXED, device=None):
    dt = torch.float64 if precision == KRR_FP64 else torch.float32
    out = torch.empty(n, r, dtype=dt, device=device or torch.device("cuda", ctx.device))
    check(lib().krr_random_block(ctx.h, n, r, col0, seed, precision, _ptr(out), out.stride(0)))
    return out


def check_gemm_args(A, B, C, ta, tb, cuda=True):
    """Shapes of a batched product C[b] = op(A[b]) op(B[b]): A (batch, M, K)
    or (batch, K, M) with ta, B (batch, K, N) or (batch, N, K) with tb, C
    None or (batch, M, N); every tensor 3-D, contiguous float32 (CUDA when
    cuda).  Returns (batch, M, N, K); raises ValueError otherwise."""
    for t, name in ((A, "A"), (B, "B"), (C, "C")):
        if t is None and name == "C":
            continue
        if t.dim() != 3 or t.dtype != torch.float32 or (cuda and not t.is_cuda):
            raise ValueError("%s must be a 3-D %sfloat32 tensor" % (name, "CUDA " if cuda else ""))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    batch = A.shape[0]
    M, K = (A.shape[2], A.shape[1]) if ta else (A.shape[1], A.shape[2])
    KB, N = (B.shape[2], B.shape[1]) if tb else (B.shape[1], B.shape[2])
    if B.shape[0] != batch or KB != K:
        raise ValueError("krr_gemm_f32_batched: A and B do not conform")
    if C is not None and tuple(C.shape) != (batch, M, N):
        raise ValueError("krr_gemm_f32_batched: C must be (batch, M, N)")
    tiles = batch * -(-M // 128) * -(-N // 128)
    if max(batch, M, N, K, tiles) > 0x7FFFFFFF:
        raise ValueError("krr_gemm_f32_batched: sizes or the count of 128 x 128 output tiles above 2^31 - 1")
    return batch, M, N, K


def krr_gemm_f32_batched(ctx, A, B, C=None, alpha=1.0, beta=0.0, ta=False, tb=False, path=0):
    """C[b] = alpha op(A[b]) op(B[b]) + beta C[b] for 3-D contiguous float32
    CUDA tensors: A (batch, M, K), or (batch, K, M) with ta; B (batch, K, N),
    or (batch, N, K) with tb; C (batch, M, N), allocated when None.  path: 0
    library's choice, 1 tensor cores (three TF32 products), 2 CUDA cores."""
    batch, M, N, K = check_gemm_args(A, B, C, ta, tb)
    if C is None:
        C = torch.zeros(batch, M, N, dtype=torch.float32, device=A.device)
    check(lib().krr_gemm_f32_batched(ctx.h, batch, M, N, K, float(alpha), _ptr(A), A.shape[2], A.stride(0),
                                     int(bool(ta)), _ptr(B), B.shape[2], B.stride(0), int(bool(tb)), float(beta),
                                     _ptr(C), N, C.stride(0), int(path)))
    return C


def krr_h_partition(left, right, lo, hi, eta):
    """Near and far blocks of an H matrix over a postorder cluster tree
    (host arrays: left / right int32[n_nodes], lo / hi float64
    n_nodes x d); returns (near, far), int32 arrays of node pairs (k x 2)
    in the library's depth-first order."""
    import numpy as np
    left = np.ascontiguousarray(left, dtype=np.int32)
    right = np.ascontiguousarray(right, dtype=np.int32)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    nn = left.shape[0]
    if left.ndim != 1 or right.shape != (nn,) or lo.ndim != 2 or lo.shape[0] != nn or hi.shape != lo.shape:
        raise ValueError("krr_h_partition: left, right int32[n_nodes]; lo, hi float64 n_nodes x d")
    cn, cf = 4 * nn, 4 * nn
    while True:
        near = np.empty((cn, 2), np.int32)
        far = np.empty((cf, 2), np.int32)
        n_near, n_far = ctypes.c_int64(0), ctypes.c_int64(0)
        code = lib().krr_h_partition(nn, left.ctypes.data, right.ctypes.data, lo.shape[1], lo.ctypes.data,
                                     hi.ctypes.data, float(eta), near.ctypes.data, cn, ctypes.byref(n_near),
                                     far.ctypes.data, cf, ctypes.byref(n_far))
        if code != 0 and (n_near.value > cn or n_far.value > cf):
            cn, cf = max(cn, n_near.value), max(cf, n_far.value)
            continue
        check(code)
        return near[:n_near.value].copy(), far[:n_far.value].copy()


def krr_one_vs_all(ctx, cls, c):
    """n x c float64 right-hand sides of the c one-vs-all problems."""
    _need(cls, torch.int32, "cls", dims=1)
    cls = cls.contiguous()
    Y = torch.empty(cls.shape[0], c, dtype=torch.float64, device=cls.device)
    check(lib().krr_one_vs_all(ctx.h, _ptr(cls), cls.shape[0], c, _ptr(Y), c))
    return Y


def default_options(**kw):
    o = _lib.krr_options()
    lib().krr_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, "lam" if k == "lambda_" else k, v)
    return o


class HSS:
    """Owner of a krr_hss handle."""

    def __init__(self, ctx, handle, n):
        self.ctx, self.h, self.n = ctx, handle, n
        ctx._handles.add(self)

    def factor(self):
        check(lib().hss_factor(self.h))

    def update_lambda(self, lam):
        check(lib().hss_update_lambda(self.h, lam))

    def solve(self, y, tol=0.0, max_refine=100, raise_on_no_convergence=True):
        """alpha (n x nrhs float64, original order) and the final residual.
        With raise_on_no_convergence=False a solve that stops above tol
        returns its last iterate and residual instead of raising."""
        _need(y, torch.float64, "y")
        y = y.contiguous()
        alpha = torch.empty(y.shape, dtype=torch.float64, device=y.device)
        res = ctypes.c_double(-1.0)
        code = lib().hss_solve(self.h, _ptr(y), y.shape[1], y.shape[1], _ptr(alpha), alpha.shape[1], tol,
                               max_refine, ctypes.byref(res))
        if code != _lib.KRR_ERR_NO_CONVERGENCE or raise_on_no_convergence:
            check(code)
        return alpha, res.value

    def predict_classes(self, Xt, alpha, absolute=False):
        """One-vs-all classes (argmax of the c decision values) and the
        decision values: (labels int32 [m], dec float64 m x c)."""
        _need(Xt, torch.float32, "Xt")
        _need(alpha, torch.float64, "alpha")
        m, c = Xt.shape[0], alpha.shape[1]
        dec = torch.empty(m, c, dtype=torch.float64, device=Xt.device)
        lab = torch.empty(m, dtype=torch.int32, device=Xt.device)
        check(lib().krr_predict_classes(self.h, _ptr(Xt.contiguous()), m, _ptr(alpha), c, alpha.stride(0),
                                        1 if absolute else 0, _ptr(dec), c, _ptr(lab)))
        return lab, dec

    def matvec(self, x):
        """y = H x with the compressed HSS matrix H (x: n x nrhs float64,
        original order)."""
        _need(x, torch.float64, "x")
        if x.shape[0] != self.n:
            raise ValueError("x must have n = %d rows" % self.n)
        x = x.contiguous()
        y = torch.empty_like(x)
        check(lib().hss_matvec(self.h, _ptr(x), x.shape[1], x.shape[1], _ptr(y), y.shape[1]))
        return y

    def predict(self, Xt, alpha):
        _need(Xt, torch.float32, "Xt")
        _need(alpha, torch.float64, "alpha")
        out = torch.empty(Xt.shape[0], alpha.shape[1], dtype=torch.float64, device=Xt.device)
        check(lib().krr_predict(self.h, _ptr(Xt), Xt.shape[0], _ptr(alpha), alpha.shape[1], alpha.stride(0),
                                _ptr(out), out.stride(0)))
        return out

    def heldout_grad(self, Xt, y, yt, tol=1e-6, max_refine=200, grad=True, want_alpha=False):
        """krr_heldout_grad: {"loss", "dh", "dlambda", "dX" (n x d float64,
        original order), "alpha", "resid"}; without grad only the loss."""
        _need(Xt, torch.float32, "Xt")
        y = y.reshape(-1).contiguous()
        yt = yt.reshape(-1).contiguous()
        _need(y, torch.float64, "y", dims=1)
        _need(yt, torch.float64, "yt", dims=1)
        d = Xt.shape[1]
        loss, dh, dl, res = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double(-1.0)
        dX = torch.empty(self.n, d, dtype=torch.float64, device=Xt.device) if grad else None
        alpha = torch.empty(self.n, dtype=torch.float64, device=Xt.device) if want_alpha else None
        check(lib().krr_heldout_grad(self.h, _ptr(Xt.contiguous()), Xt.shape[0], _ptr(y), _ptr(yt), tol, max_refine,
                                     ctypes.byref(loss), ctypes.byref(dh) if grad else None,
                                     ctypes.byref(dl) if grad else None, _ptr(dX), d, _ptr(alpha),
                                     ctypes.byref(res)))
        out = {"loss": loss.value, "resid": res.value, "alpha": alpha}
        if grad:
            out.update(dh=dh.value, dlambda=dl.value, dX=dX)
        return out

    def stats(self):
        st = _lib.krr_hss_stats()
        check(lib().hss_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def permutation(self):
        p = lib().hss_permutation(self.h)
        return p

    def close(self):
        if getattr(self, "h", None):
            # after its context's close the handle is already gone
            if not _shutting_down[0] and getattr(self.ctx, "h", None):
                lib().hss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedHSS(HSS):
    """A handle over many problems (hss_compress_batched)."""

    def __init__(self, ctx, handle, n, offsets):
        super().__init__(ctx, handle, n)
        self.offsets = offsets

    def predict(self, Xt, alpha, test_offsets):
        _need(Xt, torch.float32, "Xt")
        _need(alpha, torch.float64, "alpha")
        toff, toffp = _i64_array(test_offsets)
        out = torch.empty(Xt.shape[0], alpha.shape[1], dtype=torch.float64, device=Xt.device)
        check(lib().krr_predict_batched(self.h, _ptr(Xt), Xt.shape[0], toffp, _ptr(alpha), alpha.shape[1],
                                        alpha.stride(0), _ptr(out), out.stride(0)))
        return out


def hss_compress_batched(ctx, X, offsets, h, opts):
    """One handle for the block-diagonal system of many problems: rows
    [offsets[p], offsets[p+1]) of X with Gaussian width h[p]."""
    import numpy as np
    _need(X, torch.float32, "X")
    n, d = X.shape
    off, offp = _i64_array(offsets)
    hw = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
    hnd = ctypes.c_void_p()
    check(lib().hss_compress_batched(ctx.h, _ptr(X), n, d, len(off) - 1, offp, hw.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(opts), ctypes.byref(hnd)))
    return BatchedHSS(ctx, hnd, n, off)


def hss_compress(ctx, X, opts):
    _need(X, torch.float32, "X")
    n, d = X.shape
    h = ctypes.c_void_p()
    check(lib().hss_compress(ctx.h, _ptr(X), n, d, ctypes.byref(opts), ctypes.byref(h)))
    return HSS(ctx, h, n)


class HeldOutLoss(torch.autograd.Function):
    """L(X, h, lambda) = 1/2 ||K(Xt, X) alpha - yt||^2 with
    alpha = (K + lambda I)^{-1} y, through an HSS solve.

    forward compresses K + lambda I at (X, h, lambda) and calls
    krr_heldout_grad, which also evaluates the adjoint gradient when any of
    X, h, lambda requires it; backward scales that gradient by the incoming
    one.  h and lambda are 0-dim tensors (or floats, then not
    differentiated)."""

    @staticmethod
    def forward(fctx, X, h, lam, Xt, y, yt, kctx, opts, tol, max_refine):
        import copy
        o = copy.copy(opts)
        o.h = float(h)
        o.lam = float(lam)
        want = any(fctx.needs_input_grad[:3])
        H = hss_compress(kctx, X.detach().contiguous(), o)
        try:
            r = H.heldout_grad(Xt.detach(), y.detach().to(torch.float64), yt.detach().to(torch.float64), tol,
                               max_refine, grad=want)
        finally:
            H.close()
        dev = X.device
        if want:
            fctx.save_for_backward(r["dX"], torch.tensor(r["dh"], dtype=torch.float64, device=dev),
                                   torch.tensor(r["dlambda"], dtype=torch.float64, device=dev))
        fctx.h_is_tensor = torch.is_tensor(h)
        fctx.lam_is_tensor = torch.is_tensor(lam)
        return torch.tensor(r["loss"], dtype=torch.float64, device=dev)

    @staticmethod
    def backward(fctx, gout):
        dX, dh, dl = fctx.saved_tensors
        gX = (gout * dX).to(torch.float32) if fctx.needs_input_grad[0] else None
        gh = (gout * dh) if fctx.h_is_tensor and fctx.needs_input_grad[1] else None
        gl = (gout * dl) if fctx.lam_is_tensor and fctx.needs_input_grad[2] else None
        return gX, gh, gl, None, None, None, None, None, None, None


def krr_heldout_loss(ctx, X, h, lam, Xt, y, yt, opts=None, tol=1e-6, max_refine=200):
    """Differentiable held-out loss (see HeldOutLoss)."""
    if opts is None:
        opts = default_options()
    return HeldOutLoss.apply(X, h, lam, Xt, y, yt, ctx, opts, tol, max_refine)
