"""Tensor-core pair kernel (integer points: counts and interaction sums) against the CPU
oracle (counts bit-exact, FP64 sums within 1e-5), through the C ABI.

The device takes the TF32 tensor-core form only while the absolute values of its eight
terms sum to less than 2^24 (then every partial sum is an exact FP32 integer). These
tests check that the mode is chosen exactly on that side of the bound, that counts are
bit-exact at the largest admitted coordinates (near-ties, every term at its maximum),
in the degenerate all-hit case, on ragged sizes that span many tiles, and that the
bounded waits of the kernel end it with CC_ERR_TIMEOUT when no copy arrives.
"""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TC_MIN_N = 8192


@pytest.fixture(scope="module")
def cc():
    import paper_1901_11204_gb300 as cc
    cc.build()
    cc.lib()
    return cc


def dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def gpu_count(cc, x, y, z, r2):
    t = dev(x, y, z)
    out = cc.count_pairs(*t, r2=r2)
    torch.cuda.synchronize()
    return cc.as_u64(out), cc.stream_mode()


def fp32_pipe_count(cc, x, y, z, r2):
    """The same count through the no-allocation entry point, which always runs the
    FP32-pipe kernel (an independent GPU implementation of the same predicate)."""
    t = dev(x, y, z)
    out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    pts = cc.cc_points(cc.CC_I32, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), None)
    st = cc.lib().cc_count_pairs_noalloc(ctypes.byref(pts), len(x), r2, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == cc.CC_OK
    torch.cuda.synchronize()
    return cc.as_u64(out)


def tc_exact(m, r2e):
    """The device's admission test for the tensor-core form (sum of term bounds < 2^24)."""
    c = max(r2e + 1, 3 * m * m)
    return 9 * m * m + c + (1 << 22) + 2048 < (1 << 24)


def box_points(rng, n, span):
    return [rng.integers(0, span + 1, n).astype(np.int32) for _ in range(3)]


def corner_near_ties(rng, n, span, r2):
    """Points crowded at the eight corners of [0, span]^3 (largest |centred coordinate|,
    so every product term of the contraction is near its maximum), each base point with
    partners at squared distance r2 - 1, r2 and r2 + 1 pointing into the box, plus exact
    duplicates."""
    deltas = {}
    lim = int(np.ceil(np.sqrt(r2 + 1))) + 1
    for dx in range(0, lim + 1):
        for dy in range(0, lim + 1):
            for dz in range(0, lim + 1):
                d2 = dx * dx + dy * dy + dz * dz
                if d2 in (r2 - 1, r2, r2 + 1):
                    deltas.setdefault(d2, []).append((dx, dy, dz))
    assert all(k in deltas for k in (r2 - 1, r2, r2 + 1)), deltas.keys()
    pts = []
    while len(pts) < n:
        corner = rng.integers(0, 2, 3)
        base = np.where(corner == 0, rng.integers(0, 6, 3), span - rng.integers(0, 6, 3))
        sgn = np.where(corner == 0, 1, -1)
        pts.append(base.copy())
        for d2 in (r2 - 1, r2, r2 + 1):
            d = np.array(deltas[d2][rng.integers(0, len(deltas[d2]))])
            pts.append(base + sgn * d)
        if rng.random() < 0.2:
            pts.append(base.copy())
    a = np.array(pts[:n], dtype=np.int64)
    assert a.min() >= 0 and a.max() <= span
    a = a[rng.permutation(n)]
    return [np.ascontiguousarray(a[:, k]).astype(np.int32) for k in range(3)]


def test_mode_boundary_small_r2(cc):
    """Half-span 1023 (span 2046) is the largest admitted for small r2; 1024 is not."""
    assert tc_exact(1023, 9) and not tc_exact(1024, 9)
    rng = np.random.default_rng(7)
    for span, want in ((2046, cc.MODE_TENSOR), (2047, cc.MODE_FP32_EXACT)):
        x, y, z = box_points(rng, 20000, span)
        x[0], y[0], z[0] = 0, 0, 0
        x[1], y[1], z[1] = span, span, span
        got, mode = gpu_count(cc, x, y, z, 9)
        assert mode == want, (span, mode)
        assert got == oracle.count_i32(x, y, z, 9)


def test_mode_boundary_large_r2(cc):
    """For large r2 the |n_i - r2e - 1| term decides: both sides of the bound at m = 1000."""
    m = 1000
    r2_max = max(r for r in range(3_500_000, 3_700_000) if tc_exact(m, r))
    rng = np.random.default_rng(8)
    x, y, z = box_points(rng, 16500, 2 * m)
    x[0], y[0], z[0] = 0, 0, 0
    x[1], y[1], z[1] = 2 * m, 2 * m, 2 * m
    for r2, want in ((r2_max, cc.MODE_TENSOR), (r2_max + 1, cc.MODE_FP32_EXACT)):
        got, mode = gpu_count(cc, x, y, z, r2)
        assert mode == want, (r2, mode)
        assert got == oracle.count_i32(x, y, z, r2)


@pytest.mark.parametrize("r2", [1, 50, 301])
def test_near_ties_at_the_range_limit(cc, r2):
    rng = np.random.default_rng(100 + r2)
    x, y, z = corner_near_ties(rng, 24001, 2046, r2)
    x[0], y[0], z[0] = 0, 0, 0            # span exactly 2046: centred coordinates reach +-1023
    x[1], y[1], z[1] = 2046, 2046, 2046
    got, mode = gpu_count(cc, x, y, z, r2)
    assert mode == cc.MODE_TENSOR
    want = oracle.count_i32(x, y, z, r2)
    assert got == want
    assert got == fp32_pipe_count(cc, x, y, z, r2)


def test_all_points_identical(cc):
    n = 20001
    x = np.full(n, 17, np.int32)
    got, mode = gpu_count(cc, x, x.copy(), x.copy(), 0)
    assert mode == cc.MODE_TENSOR
    assert got == n * (n - 1) // 2


@pytest.mark.parametrize("n", [8192, 8193, 16384, 16385, 16511, 16512, 16513, 33025, 65791])
def test_ragged_sizes(cc, n):
    rng = np.random.default_rng(n)
    x, y, z = box_points(rng, n, 1023)
    got, mode = gpu_count(cc, x, y, z, 400)
    assert mode == cc.MODE_TENSOR
    assert got == oracle.count_i32(x, y, z, 400)


def test_below_threshold_uses_fp32_pipe(cc):
    rng = np.random.default_rng(3)
    x, y, z = box_points(rng, TC_MIN_N - 1, 1023)
    got, mode = gpu_count(cc, x, y, z, 400)
    assert mode == cc.MODE_FP32_EXACT
    assert got == oracle.count_i32(x, y, z, 400)


SUM_RTOL = 1e-5


def gpu_sum(cc, x, y, z, r2):
    t = dev(x, y, z)
    s, c = cc.interaction_sum(*t, r2=r2)
    torch.cuda.synchronize()
    return float(s.item()), cc.as_u64(c), cc.stream_mode()


@pytest.mark.parametrize("n,r2", [(TC_MIN_N, 4), (TC_MIN_N + 5, 400), (20001, 2000)])
def test_sums_on_tensor_cores(cc, n, r2):
    """Interaction sums take the tensor-core kernel too: count bit-exact, sum within
    1e-5 of the oracle's FP64 sum and of the FP32-pipe kernel's sum."""
    rng = np.random.default_rng(n + r2)
    x, y, z = box_points(rng, n, 160)
    s, c, mode = gpu_sum(cc, x, y, z, r2)
    assert mode == cc.MODE_TENSOR
    want_c, want_s = oracle.sum_i32(x, y, z, r2)
    assert c == want_c == oracle.count_i32(x, y, z, r2)
    assert abs(s - want_s) <= SUM_RTOL * want_s
    cc.set_tensor_cores(False)
    try:
        s2, c2, mode2 = gpu_sum(cc, x, y, z, r2)
    finally:
        cc.set_tensor_cores(True)
    assert mode2 == cc.MODE_FP32_EXACT and c2 == c
    assert abs(s - s2) <= SUM_RTOL * want_s


def test_sums_near_ties_at_the_range_limit(cc):
    rng = np.random.default_rng(150)
    x, y, z = corner_near_ties(rng, 24001, 2046, 50)
    x[0], y[0], z[0] = 0, 0, 0
    x[1], y[1], z[1] = 2046, 2046, 2046
    s, c, mode = gpu_sum(cc, x, y, z, 50)
    assert mode == cc.MODE_TENSOR
    want_c, want_s = oracle.sum_i32(x, y, z, 50)
    assert c == want_c
    assert abs(s - want_s) <= SUM_RTOL * want_s


def test_sums_all_points_identical(cc):
    """Every pair hits at d = 0: each term is 1/1e-6."""
    n = 20001
    x = np.full(n, 17, np.int32)
    s, c, mode = gpu_sum(cc, x, x.copy(), x.copy(), 0)
    assert mode == cc.MODE_TENSOR
    assert c == n * (n - 1) // 2
    want = c / 1e-6
    assert abs(s - want) <= SUM_RTOL * want


@pytest.mark.parametrize("frac", [0.0, 0.5, 0.95])
def test_clustered_sets(cc, frac):
    """A dense cluster inside a wide bounding box (the device then takes the in-register
    count form; uniform sets take the walk form): exact either way."""
    rng = np.random.default_rng(int(frac * 100) + 40)
    n = 20001
    x, y, z = box_points(rng, n, 1023)
    k = int(frac * n)
    for a in (x, y, z):
        a[:k] = 500 + rng.integers(0, 24, k)
    p = rng.permutation(n)
    x, y, z = x[p], y[p], z[p]
    got, mode = gpu_count(cc, x, y, z, 9)
    assert mode == cc.MODE_TENSOR
    assert got == oracle.count_i32(x, y, z, 9)
    assert got == fp32_pipe_count(cc, x, y, z, 9)


def test_tc_bounded_wait_timeout(cc):
    """No copy is issued: the MMA lane's wait runs out, every role stops, TMEM is freed,
    the count reads CC_COUNT_INVALID (the sum NaN), the status CC_ERR_TIMEOUT, and the
    next call is correct."""
    rng = np.random.default_rng(11)
    x, y, z = box_points(rng, 20000, 1023)
    t = dev(x, y, z)
    cc.set_wait_limit_ns(20_000_000)
    cc.debug_stall_copies(True)
    try:
        out = cc.count_pairs(*t, r2=9)
        assert cc.stream_status() == cc.CC_ERR_TIMEOUT
        assert cc.stream_mode() == cc.MODE_TENSOR
        assert cc.as_u64(out) == cc.CC_COUNT_INVALID
        s, c = cc.interaction_sum(*t, r2=9)
        assert cc.stream_status() == cc.CC_ERR_TIMEOUT
        assert cc.as_u64(c) == cc.CC_COUNT_INVALID
        assert np.isnan(float(s.item()))
    finally:
        cc.debug_stall_copies(False)
        cc.set_wait_limit_ns(2_000_000_000)
    got, mode = gpu_count(cc, x, y, z, 9)
    assert mode == cc.MODE_TENSOR
    assert got == oracle.count_i32(x, y, z, 9)
    assert cc.stream_status() == cc.CC_OK


@pytest.mark.parametrize("r2", [9, 400])
def test_switch_between_kernels_gives_equal_counts(cc, r2):
    """cc_set_tensor_cores(0) sends the same call to the FP32-pipe kernel: equal counts."""
    import synth
    c = synth.cfg2(70001)
    t = dev(c["x"], c["y"], c["z"])
    out = cc.count_pairs(*t, r2=r2)
    torch.cuda.synchronize()
    assert cc.stream_mode() == cc.MODE_TENSOR
    a = cc.as_u64(out)
    cc.set_tensor_cores(False)
    try:
        out = cc.count_pairs(*t, r2=r2)
        torch.cuda.synchronize()
        assert cc.stream_mode() == cc.MODE_FP32_EXACT
        b = cc.as_u64(out)
    finally:
        cc.set_tensor_cores(True)
    assert a == b == oracle.count_i32(c["x"], c["y"], c["z"], r2)


def test_two_streams_interleaved_stress(cc):
    """Tensor-core counts and sums on two streams at once, interleaved with small-set
    calls, many times over: every result exact and no device-side wait runs out (a stall
    anywhere in a kernel's pipeline would surface as CC_ERR_TIMEOUT after the wait bound)."""
    rng = np.random.default_rng(41)
    big = [box_points(rng, n, 1023) for n in (9001, 20000, 40001)]
    want = [oracle.count_i32(*b, 9) for b in big]
    small = box_points(rng, 3000, 40)
    want_small = oracle.count_i32(*small, 9)
    tb = [dev(*b) for b in big]
    ts = dev(*small)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for rep in range(40):
        for k, s in enumerate(streams):
            with torch.cuda.stream(s):
                j = (rep + k) % 3
                outs.append((cc.count_pairs(*tb[j], r2=9, stream=s), want[j]))
                outs.append((cc.count_pairs(*ts, r2=9, stream=s), want_small))
                if rep % 8 == k:
                    sm, c = cc.interaction_sum(*tb[j], r2=9, stream=s)
                    outs.append((c, want[j]))
    torch.cuda.synchronize()
    for s in streams:
        assert cc.stream_status(s) == cc.CC_OK
    assert [cc.as_u64(o) for o, _ in outs] == [w for _, w in outs]
