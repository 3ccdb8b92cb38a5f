"""The C-ABI library builds, loads, and exports every symbol include/lsk.h
declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_02798_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lsk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsk_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_path():
    names = declared_functions()
    for want in ["lsk_cs_sketch", "lsk_gauss_sketch", "lsk_gram", "lsk_rownorms_prod",
                 "lsk_leverage_scores", "lsk_sketch_precondition_lsq", "lsk_sketch_qr"]:
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    from paper_2203_02798_gb300 import LsqOpts
    o = LsqOpts()
    lib.lsk_lsq_default_opts.argtypes = [ctypes.POINTER(LsqOpts), ctypes.c_int64]
    lib.lsk_lsq_default_opts(ctypes.byref(o), 64)
    assert o.r == 64 * 64 and o.k == 128 and o.tol == 1e-10
    # a NULL context is rejected on the host before any CUDA call
    for name in ["lsk_cs_sketch", "lsk_gram", "lsk_leverage_scores", "lsk_sync"]:
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
    lib.lsk_sync.argtypes = [ctypes.c_void_p]
    assert lib.lsk_sync(None) == -1
    lib.lsk_error_string.restype = ctypes.c_char_p
    lib.lsk_error_string.argtypes = [ctypes.c_void_p]
    assert lib.lsk_error_string(None) == b"null context"


def test_binding_exports_same_names():
    import paper_2203_02798_gb300 as p
    for n in ["cs_sketch", "gauss_sketch", "gram", "rownorms_prod", "leverage_scores",
              "sketch_precondition_lsq", "sketch_qr", "debug_hash", "debug_gauss"]:
        assert callable(getattr(p, n))


def test_fused_sketch_switch_is_host_state(lib):
    """lsk_set_fused_sketch only sets process-wide host state (no CUDA call):
    mode 1 (fused where the shape favours it) by default, values clamped to
    [0, 2], returns the previous mode."""
    lib.lsk_set_fused_sketch.restype = ctypes.c_int
    lib.lsk_set_fused_sketch.argtypes = [ctypes.c_int]
    assert lib.lsk_set_fused_sketch(2) == 1
    assert lib.lsk_set_fused_sketch(0) == 2
    assert lib.lsk_set_fused_sketch(7) == 0
    assert lib.lsk_set_fused_sketch(-3) == 2
    assert lib.lsk_set_fused_sketch(1) == 0
