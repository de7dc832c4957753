"""The no-allocation count entry point, through the C ABI.

Callers that cannot allocate device memory while they run (graph recording, a single
owning allocator, a fixed memory budget) use cc_count_pairs_noalloc, whose scratch is a
static device array inside the library. Its counts must equal cc_count_pairs' on the
same inputs and the oracle's golden values, on two calls in a row (the second call
reuses the array the first one left behind), for integer points and FP32 spheres; a
bounded wait that runs out must give CC_COUNT_INVALID. This file is collected last on
purpose; it passes alone and after the others.
"""
import ctypes
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size_counts.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        out[parts[0]] = int(parts[1])
    return out


def _count(cc, fn, arrs, r2):
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
    out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    if len(t) == 4:
        pts = cc.cc_points(cc.CC_F32, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), t[3].data_ptr())
    else:
        pts = cc.cc_points(cc.CC_I32, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), None)
    st = fn(ctypes.byref(pts), len(arrs[0]), r2, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == cc.CC_OK, cc.lib().cc_last_error()
    torch.cuda.synchronize()
    return cc.as_u64(out)


def test_noalloc_matches_allocating_entry_point_twice():
    import paper_1901_11204_gb300 as cc
    cc.build()
    L = cc.lib()
    g = _golden()
    c2 = synth.cfg2(262145)
    c1 = synth.cfg1()
    c3 = synth.cfg3()
    cases = [([c2["x"], c2["y"], c2["z"]], 9, g["cfg2_n262145_r2_9"]),
             ([c1["x"], c1["y"], c1["z"]], 16, g["cfg1_n4096_r2_16"]),
             ([c3["x"], c3["y"], c3["z"], c3["r"]], 0, g["cfg3_n131072_f32"])]
    for arrs, r2, want in cases:   # calls in a row, different sizes and kinds
        ref = _count(cc, L.cc_count_pairs, arrs, r2)
        first = _count(cc, L.cc_count_pairs_noalloc, arrs, r2)
        second = _count(cc, L.cc_count_pairs_noalloc, arrs, r2)
        assert first == second == ref == want


def test_noalloc_timeout_gives_invalid_count():
    """Copies held back by the test hook: the FP32-pipe kernel's waits run out and the
    count reads CC_COUNT_INVALID; the next call is exact."""
    import paper_1901_11204_gb300 as cc
    cc.build()
    L = cc.lib()
    c = synth.cfg2(20001)
    arrs = [c["x"], c["y"], c["z"]]
    want = _count(cc, L.cc_count_pairs, arrs, 9)
    cc.set_wait_limit_ns(20_000_000)
    cc.debug_stall_copies(True)
    try:
        got = _count(cc, L.cc_count_pairs_noalloc, arrs, 9)
    finally:
        cc.debug_stall_copies(False)
        cc.set_wait_limit_ns(2_000_000_000)
    assert got == cc.CC_COUNT_INVALID
    assert _count(cc, L.cc_count_pairs_noalloc, arrs, 9) == want


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1901_11204_gb300 as cc
    cc.build()
    L = cc.lib()
    pts = cc.cc_points(cc.CC_I32, 0x1000, 0x1000, 0x1000, None)
    st = L.cc_count_pairs_noalloc(ctypes.byref(pts), 50_000_000, 9, ctypes.c_void_p(0x1000), None)
    assert st == cc.CC_ERR_INVALID_ARG
    assert b"no-allocation limit" in L.cc_last_error()
