"""The C-ABI library loads, exports every entry point include/cc.h declares, and rejects
bad arguments on the host (no GPU needed for any of this)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cc():
    import paper_1901_11204_gb300 as cc
    cc.build()
    cc.lib()
    return cc


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cc_count_pairs", "cc_count_pairs_batched", "cc_interaction_sum"):
        assert must in names


def test_every_declared_symbol_is_exported(cc):
    L = ctypes.CDLL(cc.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_header(cc):
    from paper_1901_11204_gb300 import _SIGS
    assert set(_SIGS) == set(declared_functions())


def test_version_and_status_strings(cc):
    assert "sm_103a" in cc.version()
    L = cc.lib()
    assert L.cc_status_string(0) == b"CC_OK"
    assert L.cc_status_string(2) == b"CC_ERR_RANGE"


def test_host_side_argument_errors(cc):
    L = cc.lib()
    d = ctypes.c_void_p(0x1000)
    assert L.cc_count_pairs(None, 10, 0, d, None) == cc.CC_ERR_INVALID_ARG
    pts = cc.cc_points(7, 0x1000, 0x1000, 0x1000, None)
    assert L.cc_count_pairs(ctypes.byref(pts), 10, 0, d, None) == cc.CC_ERR_INVALID_ARG
    pts = cc.cc_points(cc.CC_I32, 0x1000, 0x1000, 0x1000, None)
    assert L.cc_count_pairs(ctypes.byref(pts), -1, 0, d, None) == cc.CC_ERR_INVALID_ARG
    assert L.cc_count_pairs(ctypes.byref(pts), 10, 0, None, None) == cc.CC_ERR_INVALID_ARG
    assert b"d_count" in L.cc_last_error()
    mis = cc.cc_points(cc.CC_I32, 0x1001, 0x1000, 0x1000, None)
    assert L.cc_count_pairs(ctypes.byref(mis), 10, 0, d, None) == cc.CC_ERR_INVALID_ARG
    f32 = cc.cc_points(cc.CC_F32, 0x1000, 0x1000, 0x1000, None)
    assert L.cc_interaction_sum(ctypes.byref(f32), 10, 0, d, None, None) == cc.CC_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert L.cc_plan_create(ctypes.byref(h), None, 0, 10) == cc.CC_ERR_INVALID_ARG
    assert L.cc_plan_create(ctypes.byref(h), b'{"bands": [{"n_max": 10, "r": 8, "sc": 4}]}', 10, 10) \
        == cc.CC_ERR_INVALID_ARG
    assert L.cc_plan_create(ctypes.byref(h), b'{"nothing": 1}', 10, 10) == cc.CC_ERR_INVALID_ARG
    assert L.cc_server_create(ctypes.byref(h), 0, 4) == cc.CC_ERR_INVALID_ARG
    assert L.cc_server_create(ctypes.byref(h), 1 << 20, 0) == cc.CC_ERR_INVALID_ARG


def test_no_cpu_fallback_in_product_package():
    """The product package never imports the oracle (the CPU reference is test-only)."""
    pkg = os.path.join(ROOT, "paper_1901_11204_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(dp, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "cc_oracle" not in src, f


def test_bounds_microbenchmark_compiles():
    """The tool that measures the tensor-core kernel's bounds (TMEM reads, MMA issue, the
    accumulator hand-over loop) cross-compiles for sm_103a from the committed sources."""
    from paper_1901_11204_gb300.microbench import __main__ as microbench
    exe = microbench.build()
    assert os.path.isfile(exe) and os.path.getsize(exe) > 0
