"""ctypes binding of libkrrhss.so: argument marshalling only.

Every function here forwards to the C entry point of the same name in
include/krrhss.h; device buffers are torch CUDA tensors, whose data
pointers are passed through.  The library is loaded from this directory
and never replaced by a Python or CPU implementation: if it is missing
or cannot load, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkrrhss.so")

KRR_OK = 0
KRR_ERR_NO_CONVERGENCE = 9
STATUS = {0: "KRR_OK", 1: "KRR_ERR_INVALID_ARG", 2: "KRR_ERR_NONFINITE_INPUT", 3: "KRR_ERR_OOM",
          4: "KRR_ERR_SINGULAR", 5: "KRR_ERR_RANK_BUDGET", 6: "KRR_ERR_TIMEOUT", 7: "KRR_ERR_CUDA",
          8: "KRR_ERR_NOT_IMPLEMENTED", 9: "KRR_ERR_NO_CONVERGENCE"}
KRR_TRUNCATE_AT_RMAX = 1
KRR_LAMBDA_TOL = 2
KRR_MIXED, KRR_FP64, KRR_MIXED_F64 = 0, 1, 2
KRR_ORDER_TWO_MEANS, KRR_ORDER_NATURAL, KRR_ORDER_KD, KRR_ORDER_PCA = 0, 1, 2, 3

P = ctypes.c_void_p
i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double


class krr_allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(P, ctypes.c_size_t, P)),
                ("free", ctypes.CFUNCTYPE(None, P, P)),
                ("user", P)]


class krr_tree_arrays(ctypes.Structure):
    _fields_ = [(k, ctypes.POINTER(i32)) for k in ("begin", "end", "left", "right", "parent", "level")]


class krr_options(ctypes.Structure):
    _fields_ = [("h", f64), ("lam", f64), ("eps_c", f64), ("eps_abs", f64), ("leaf", i32), ("r0", i32),
                ("p", i32), ("r_max", i32), ("seed", u64), ("precision", i32), ("flags", i32), ("ordering", i32),
                ("pad", i32)]


class krr_hss_stats(ctypes.Structure):
    _fields_ = [("n", i64), ("n_nodes", i32), ("n_levels", i32), ("max_rank", i32), ("samples", i32),
                ("rounds", i32), ("refine_steps", i32), ("memory_bytes", i64), ("t_cluster_ms", f64),
                ("t_sample_ms", f64), ("t_compress_ms", f64), ("t_factor_ms", f64), ("t_solve_ms", f64),
                ("truncated", i32), ("pad", i32)]


SIGNATURES = {
    "krr_create": (i32, [ctypes.POINTER(P), ctypes.POINTER(krr_allocator), P]),
    "krr_destroy": (None, [P]),
    "krr_last_error": (ctypes.c_char_p, []),
    "krr_launch_count": (ctypes.c_longlong, []),
    "krr_sync": (i32, [P]),
    "krr_set_wait_limit": (i32, [P, i64]),
    "krr_set_autotune": (i32, [P, i32]),
    "krr_probe_rate": (i32, [P, i32, ctypes.POINTER(f64)]),
    "krr_gemm_f32_batched": (i32, [P, i32, i32, i32, i32, ctypes.c_float, P, i64, i64, i32, P, i64, i64, i32,
                                   ctypes.c_float, P, i64, i64, i32]),
    "krr_h_partition": (i32, [i32, P, P, i32, P, P, f64, P, i64, ctypes.POINTER(i64), P, i64,
                              ctypes.POINTER(i64)]),
    "krr_standardize": (i32, [P, P, i64, i32, P, i64, P, P]),
    "krr_cluster": (i32, [P, P, i64, i32, i32, u64, P, i32, krr_tree_arrays, ctypes.POINTER(i32)]),
    "krr_order": (i32, [P, P, i64, i32, i32, i32, u64, P, i32, krr_tree_arrays, ctypes.POINTER(i32)]),
    "krr_cluster_batched": (i32, [P, P, i64, i32, i32, P, i32, u64, P, i32, krr_tree_arrays,
                                  ctypes.POINTER(i32)]),
    "krr_sample": (i32, [P, P, i64, P, i64, i32, f64, f64, P, i32, i64, P, P, P, i64]),
    "krr_sample_f64": (i32, [P, P, i64, P, i64, i32, f64, f64, P, i32, i64, P, P, P, i64]),
    "krr_sample_noalloc": (i32, [P, P, i64, P, i64, i32, f64, f64, P, i32, i64, P, P, P, i64]),
    "krr_random_block": (i32, [P, i64, i32, i32, u64, ctypes.c_int, P, i64]),
    "krr_default_options": (None, [ctypes.POINTER(krr_options)]),
    "hss_compress": (i32, [P, P, i64, i32, ctypes.POINTER(krr_options), ctypes.POINTER(P)]),
    "hss_compress_batched": (i32, [P, P, i64, i32, i32, P, P, ctypes.POINTER(krr_options), ctypes.POINTER(P)]),
    "krr_predict_batched": (i32, [P, P, i64, P, P, i32, i64, P, i64]),
    "hss_update_lambda": (i32, [P, f64]),
    "hss_factor": (i32, [P]),
    "hss_solve": (i32, [P, P, i32, i64, P, i64, f64, i32, ctypes.POINTER(f64)]),
    "krr_predict": (i32, [P, P, i64, P, i32, i64, P, i64]),
    "hss_matvec": (i32, [P, P, i32, i64, P, i64]),
    "krr_one_vs_all": (i32, [P, P, i64, i32, P, i64]),
    "krr_predict_classes": (i32, [P, P, i64, P, i32, i64, i32, P, i64, P]),
    "krr_heldout_grad": (i32, [P, P, i64, P, P, f64, i32, ctypes.POINTER(f64), ctypes.POINTER(f64),
                               ctypes.POINTER(f64), P, i64, P, ctypes.POINTER(f64)]),
    "hss_stats": (i32, [P, ctypes.POINTER(krr_hss_stats)]),
    "hss_permutation": (P, [P]),
    "hss_destroy": (None, [P]),
}

_lib = None


def lib():
    """Load libkrrhss.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libkrrhss.so is not built: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class KRRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


def check(code):
    if code != KRR_OK:
        raise KRRError(code, lib().krr_last_error().decode())
    return code
