"""The C-ABI library builds for sm_103a and exports every entry point that
include/pf.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def declared_symbols():
    with open(os.path.join(ROOT, "include", "pf.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"PF_API\s+[^;(]*?\b(pf_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pf_create", "pf_destroy", "pf_pack", "pf_filter", "pf_verify",
                     "pf_compact", "pf_filter_plain", "pf_filter_verify", "pf_sync"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1910_03936_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_1910_03936_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.pf_status_string.restype = ctypes.c_char_p
    assert lib.pf_status_string(0) == b"PF_OK"
    assert lib.pf_status_string(7) == b"PF_EDATA"


def test_pack_layout_host_helper():
    import numpy as np
    from paper_1910_03936_gb300 import build
    lib = ctypes.CDLL(build.build())
    bo = np.array([0, 0, 1, 32, 33, 97, 97], dtype=np.int64)
    wo = np.zeros(7, dtype=np.int64)
    tot = ctypes.c_int64()
    rc = lib.pf_pack_layout(ctypes.c_void_p(bo.ctypes.data), ctypes.c_int64(6),
                            ctypes.c_void_p(wo.ctypes.data), ctypes.byref(tot))
    assert rc == 0
    assert wo.tolist() == [0, 0, 1, 2, 3, 5, 5] and tot.value == 5


def test_product_path_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_1910_03936_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, fn)) as f:
                    src = f.read()
                assert "oracle" not in src.replace("oracle-free", ""), fn


def test_grouped_layout_host_helper():
    """pf_pack_layout_grouped: every sequence gets its ceil(len/32) words,
    the ranges tile [0, total) without overlap, and sequences follow each
    other in the order of (E, min(ceil(len/32), 64), index)."""
    import numpy as np
    import paper_1910_03936_gb300 as pf
    rng = np.random.default_rng(3)
    n = 5000
    lens = rng.choice([0, 1, 31, 32, 33, 100, 150, 250, 2100, 4000], size=n)
    E = rng.integers(0, pf.PF_MAX_E + 1, size=n).astype(np.int16)
    bo = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=bo[1:])
    W = (lens + 31) // 32
    for Eh in (E, None):
        ws, total = pf.pf_pack_layout_grouped(bo, Eh)
        assert total == W.sum()
        key_e = Eh.astype(np.int64) if Eh is not None else np.zeros(n, dtype=np.int64)
        order = np.lexsort((np.arange(n), np.minimum(W, 64), key_e))
        expect = np.zeros(n, dtype=np.int64)
        expect[order] = np.concatenate(([0], np.cumsum(W[order])[:-1]))
        assert np.array_equal(ws, expect)
    # empty batch, falling offsets, thresholds out of range
    ws, total = pf.pf_pack_layout_grouped(np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int16))
    assert total == 0 and ws.size == 0
    with pytest.raises(pf.PFError):
        pf.pf_pack_layout_grouped(np.array([0, 5, 3], dtype=np.int64))
    with pytest.raises(pf.PFError):
        pf.pf_pack_layout_grouped(np.array([0, 5, 9], dtype=np.int64),
                                  np.array([0, pf.PF_MAX_E + 1], dtype=np.int16))
    with pytest.raises(pf.PFError):
        pf.pf_pack_layout_grouped(np.array([0, 5, 9], dtype=np.int64),
                                  np.array([-1, 0], dtype=np.int16))


def test_host_alloc_argument_checks_without_gpu():
    """pf_host_alloc and pf_host_free refuse bad arguments before touching
    CUDA."""
    import paper_1910_03936_gb300 as pf
    lib = pf.load()
    p = ctypes.c_void_p()
    assert lib.pf_host_alloc(ctypes.c_size_t(0), ctypes.byref(p)) == 1   # PF_EINVAL
    assert lib.pf_host_alloc(ctypes.c_size_t(16), None) == 1
    assert lib.pf_host_free(None) == 0
    assert lib.pf_host_free(ctypes.c_void_p(0x1000)) == 1
