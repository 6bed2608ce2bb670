"""The C-ABI library loads and exports every entry point declared in
include/krrhss.h (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

from paper_1803_10274_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "krrhss.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(krr_\w+|hss_\w+)\s*\(", txt)))


def test_header_symbols_exported():
    L = _lib.lib()
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_binding_covers_header():
    assert set(declared()) == set(_lib.SIGNATURES)


def test_no_gpu_calls_needed_for_errors():
    L = _lib.lib()
    # argument checks run before any device work
    assert L.krr_create(None, None, None) == 1
    assert b"krr_create" in L.krr_last_error()
    o = _lib.krr_options()
    L.krr_default_options(ctypes.byref(o))
    assert o.leaf == 128 and o.r0 == 64 and o.precision == 0 and abs(o.eps_c - 0.03) < 1e-15
