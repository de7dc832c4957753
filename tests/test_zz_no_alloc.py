"""The no-allocation count entry point, through the C ABI.

Callers that cannot allocate device memory while they run (graph recording, a single
owning allocator, a fixed memory budget) use cc_count_pairs_noalloc, whose scratch is a
static device array inside the library. Its counts must equal cc_count_pairs' on the
same inputs, on two calls in a row (the second call reuses the array the first one left
behind). This file is collected last on purpose; it passes alone and after the others.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _count(cc, fn, x, y, z):
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, y, z)]
    out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    pts = cc.cc_points(cc.CC_I32, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), None)
    st = fn(ctypes.byref(pts), len(x), 9, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == cc.CC_OK, cc.lib().cc_last_error()
    torch.cuda.synchronize()
    return cc.as_u64(out)


def test_noalloc_matches_allocating_entry_point_twice():
    import paper_1901_11204_gb300 as cc
    cc.build()
    L = cc.lib()
    inputs = [synth.cfg2(262145), synth.cfg1()]
    for c in inputs:   # two calls in a row, different sizes
        want = _count(cc, L.cc_count_pairs, c["x"], c["y"], c["z"])
        got = _count(cc, L.cc_count_pairs_noalloc, c["x"], c["y"], c["z"])
        assert got == want


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1901_11204_gb300 as cc
    cc.build()
    L = cc.lib()
    pts = cc.cc_points(cc.CC_I32, 0x1000, 0x1000, 0x1000, None)
    st = L.cc_count_pairs_noalloc(ctypes.byref(pts), 50_000_000, 9, ctypes.c_void_p(0x1000), None)
    assert st == cc.CC_ERR_INVALID_ARG
    assert b"no-allocation limit" in L.cc_last_error()
