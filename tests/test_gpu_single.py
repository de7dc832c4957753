"""Single-set GPU path against the CPU oracle (parity), through the C ABI.

Counts must be bit-exact; FP32 interaction sums within 1e-5 relative of the FP64 oracle.
Sizes span several tiles of every tile configuration and ragged tails, both parities.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SUM_RTOL = 1e-5
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size_counts.txt")


@pytest.fixture(scope="module")
def cc():
    import paper_1901_11204_gb300 as cc
    cc.build()
    cc.lib()
    return cc


def dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def gpu_count(cc, x, y, z, r2=0, r=None):
    t = dev(x, y, z) + (dev(r) if r is not None else [])
    out = cc.count_pairs(*t[:3], r2=r2, r=t[3] if r is not None else None)
    torch.cuda.synchronize()
    return cc.as_u64(out)


def gpu_sum(cc, x, y, z, r2=0, r=None):
    t = dev(x, y, z) + (dev(r) if r is not None else [])
    s, c = cc.interaction_sum(*t[:3], r2=r2, r=t[3] if r is not None else None)
    torch.cuda.synchronize()
    return float(s.item()), cc.as_u64(c)


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


SIZES = [0, 1, 2, 3, 4, 5, 31, 32, 33, 64, 127, 128, 129, 255, 256, 257, 1000, 1001,
         2047, 2048, 2049, 4095, 4096, 4097, 9999, 20000, 65535, 65536, 65537]


@pytest.mark.parametrize("n", SIZES)
def test_int_random_parity(cc, n):
    rng = np.random.default_rng(1000 + n)
    box = max(4, int(round((n + 1) ** (1 / 3) * 3)))
    x, y, z = (rng.integers(0, box, n).astype(np.int32) for _ in range(3))
    for r2 in (0, 9):
        assert gpu_count(cc, x, y, z, r2) == oracle.count_i32(x, y, z, r2), (n, r2)


@pytest.mark.parametrize("n", [2, 3, 33, 257, 2049, 4096, 65537])
def test_f32_random_parity(cc, n):
    x, y, z, r = synth.sphere_points(n, 77 + n, rmin=0.01, rmax=0.04)
    want_c, want_s = oracle.count_f32(x, y, z, r)
    assert gpu_count(cc, x, y, z, 0, r) == want_c
    s, c = gpu_sum(cc, x, y, z, 0, r)
    assert c == want_c
    assert rel(s, want_s) <= SUM_RTOL or (want_c == 0 and s == 0.0)


def test_cfg1_parity(cc):
    c = synth.cfg1()
    assert gpu_count(cc, c["x"], c["y"], c["z"], 16) == oracle.count_i32(c["x"], c["y"], c["z"], 16)


@pytest.mark.parametrize("n", [1, 2, 7, 64, 65, 4096, 4097, 30001])
def test_line_closed_form(cc, n):
    """x_i = permuted 0..n-1: pairs with |i-j| <= k number sum_{m<=k}(n-m) (any wrap error
    shows, because wrapped pairs have large |i-j|)."""
    rng = np.random.default_rng(n)
    x = rng.permutation(n).astype(np.int32)
    zero = np.zeros(n, dtype=np.int32)
    for k in sorted({0, 1, 3, n // 2, n}):
        want = sum(n - m for m in range(1, min(k, n - 1) + 1))
        # line spans > 2364 switch to the integer difference path, shorter ones stay fast
        assert gpu_count(cc, x, zero, zero, k * k) == want, (n, k)


def test_lattice_closed_form(cc):
    rng = np.random.default_rng(5)
    for L in [(3, 4, 5), (17, 9, 23), (40, 41, 42)]:
        x, y, z = pins.lattice_points(L, rng)
        for r2 in (0, 1, 2, 3, 5, 9):
            assert gpu_count(cc, x, y, z, r2) == pins.lattice_pairs_closed_form(L, r2), (L, r2)


@pytest.mark.parametrize("n", [262144, 262145])
def test_all_identical_full_size(cc, n):
    """Every pair collides: N(N-1)/2 (Proposition 1), at the headline size."""
    v = np.full(n, 11, dtype=np.int32)
    assert gpu_count(cc, v, v, v, 0) == n * (n - 1) // 2


def test_wide_span_parity(cc):
    """Spans beyond the fast form's exact range use the integer difference path."""
    rng = np.random.default_rng(9)
    for n, box in [(3000, 30000), (20001, 5000), (777, 32768)]:
        x, y, z = (rng.integers(0, box, n).astype(np.int32) for _ in range(3))
        for r2 in (0, 40000, 2_000_000):
            assert gpu_count(cc, x, y, z, r2) == oracle.count_i32(x, y, z, r2), (n, box, r2)


def test_huge_r2_counts_everything(cc):
    rng = np.random.default_rng(10)
    n = 5001
    x, y, z = (rng.integers(-1000, 1000, n).astype(np.int32) for _ in range(3))
    assert gpu_count(cc, x, y, z, 0xFFFFFFFF) == n * (n - 1) // 2
    x2 = x * 10
    assert gpu_count(cc, x2, y, z, 0xFFFFFFFF) == n * (n - 1) // 2


def test_range_error(cc):
    n = 100
    x = np.zeros(n, dtype=np.int32)
    x[0] = 40000
    t = dev(x, x, x)
    out = cc.count_pairs(*t, r2=1)
    st = cc.stream_status()
    assert st == cc.CC_ERR_RANGE
    assert cc.as_u64(out) == cc.CC_COUNT_INVALID
    assert cc.validate_points(*t) == cc.CC_ERR_RANGE
    ok = dev(np.arange(n, dtype=np.int32), x * 0, x * 0)
    assert cc.validate_points(*ok) == cc.CC_OK


def test_negative_and_extreme_coordinates(cc):
    rng = np.random.default_rng(11)
    n = 3001
    base = np.int32(-2_000_000_000)
    x, y, z = (base + rng.integers(0, 40, n).astype(np.int32) for _ in range(3))
    assert gpu_count(cc, x, y, z, 5) == oracle.count_i32(x, y, z, 5)


def test_f32_nan_and_ties(cc):
    n = 1001
    x = np.arange(n, dtype=np.float32)
    zero = np.zeros(n, dtype=np.float32)
    r = np.full(n, 1.5, dtype=np.float32)
    want = sum(n - m for m in range(1, 4))
    assert gpu_count(cc, x, zero, zero, 0, r) == want
    s, c = gpu_sum(cc, x, zero, zero, 0, r)
    assert c == want
    assert rel(s, sum((n - m) / m for m in range(1, 4))) <= SUM_RTOL
    x2 = x.copy()
    x2[5] = np.nan
    assert gpu_count(cc, x2, zero, zero, 0, r) == oracle.count_f32(x2, zero, zero, r)[0]


def test_int_sum_parity(cc):
    rng = np.random.default_rng(12)
    n = 5000
    x, y, z = (rng.integers(0, 30, n).astype(np.int32) for _ in range(3))
    s, c = gpu_sum(cc, x, y, z, 4)
    want_c, want_s = oracle.sum_i32(x, y, z, 4)
    assert c == want_c == oracle.count_i32(x, y, z, 4)
    assert rel(s, want_s) <= SUM_RTOL


def test_stream_and_repeat_determinism(cc):
    c = synth.cfg1()
    t = dev(c["x"], c["y"], c["z"])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = [cc.count_pairs(*t, r2=16, stream=s) for _ in range(3)]
    s.synchronize()
    vals = {cc.as_u64(o) for o in outs}
    assert len(vals) == 1


@pytest.mark.parametrize("kind", ["i32", "f32"])
def test_bounded_wait_timeout(cc, kind):
    """The FP32-pipe kernel's copy issuers hold back every copy: the warps' waits run out
    after the short limit, the kernel returns, the count reads CC_COUNT_INVALID (the sum
    NaN), the status CC_ERR_TIMEOUT, and the context still works."""
    n = 20001
    if kind == "i32":
        c = synth.cfg2(n)
        arrs, r2 = [c["x"], c["y"], c["z"]], 9
        want = oracle.count_i32(*arrs, r2)
    else:
        arrs = list(synth.sphere_points(n, 41, rmin=0.002, rmax=0.006))
        r2 = 0
        want = oracle.count_f32(*arrs)[0]
    t = dev(*arrs)
    r = t[3] if kind == "f32" else None
    cc.set_tensor_cores(False)
    cc.set_wait_limit_ns(20_000_000)
    cc.debug_stall_copies(True)
    try:
        out = cc.count_pairs(*t[:3], r2=r2, r=r)
        assert cc.stream_status() == cc.CC_ERR_TIMEOUT
        assert cc.as_u64(out) == cc.CC_COUNT_INVALID
        s, c2 = cc.interaction_sum(*t[:3], r2=r2, r=r)
        assert cc.stream_status() == cc.CC_ERR_TIMEOUT
        assert cc.as_u64(c2) == cc.CC_COUNT_INVALID
        assert np.isnan(float(s.item()))
    finally:
        cc.debug_stall_copies(False)
        cc.set_wait_limit_ns(2_000_000_000)
        cc.set_tensor_cores(True)
    # the next calls on the same stream are correct and report no error
    out = cc.count_pairs(*t[:3], r2=r2, r=r)
    torch.cuda.synchronize()
    assert cc.as_u64(out) == want
    assert cc.stream_status() == cc.CC_OK


def test_small_set_kernel_reports_range_and_recovers(cc):
    """The one-launch kernel for small sets: a span beyond 32767 gives CC_COUNT_INVALID
    and CC_ERR_RANGE; its header words are left clean, so the next small and large calls
    on the stream are exact."""
    c = synth.cfg1()
    t = dev(c["x"], c["y"], c["z"])
    bad = c["x"].copy()
    bad[17] = 40000
    tb = dev(bad, c["y"], c["z"])
    out = cc.count_pairs(*tb, r2=16)
    assert cc.stream_status() == cc.CC_ERR_RANGE
    assert cc.as_u64(out) == cc.CC_COUNT_INVALID
    assert cc.stream_mode() == cc.MODE_RANGE_ERROR
    assert gpu_count(cc, c["x"], c["y"], c["z"], 16) == oracle.count_i32(c["x"], c["y"], c["z"], 16)
    assert cc.stream_status() == cc.CC_OK
    c2 = synth.cfg2(20001)
    assert gpu_count(cc, c2["x"], c2["y"], c2["z"], 9) == oracle.count_i32(c2["x"], c2["y"], c2["z"], 9)


def _golden():
    out = {}
    if not os.path.exists(GOLDEN):
        return out
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        out[parts[0]] = (int(parts[1]), float(parts[2]) if len(parts) > 2 else None)
    return out


@pytest.mark.parametrize("n", [262144, 262145])
def test_cfg2_full_size(cc, n):
    g = _golden()
    c = synth.cfg2(n)
    key = f"cfg2_n{n}_r2_9"
    want = g[key][0] if key in g else oracle.count_i32(c["x"], c["y"], c["z"], 9)
    assert gpu_count(cc, c["x"], c["y"], c["z"], 9) == want
    s = synth.cfg2(n, same_cell=True)
    # same-cell predicate at full size: Algorithm 1 (O(N)) gives the exact answer
    assert gpu_count(cc, s["x"], s["y"], s["z"], 0) == oracle.count_colls(s["x"], s["y"], s["z"])


@pytest.mark.parametrize("n", [262144, 262145])
@pytest.mark.parametrize("tc", [True, False])
def test_cfg2_planted_full_size(cc, n, tc):
    """Headline sizes with coincident objects planted at the ends of the schedule's
    windows: the last object against the first (across the wrap) and against the far end
    of its window, the objects around (n-1)/2 and n/2 (the even-N extra step), on the
    tensor-core kernel and on the FP32 pipe; the count must equal the oracle's golden."""
    g = _golden()
    p = synth.cfg2_planted(n)
    key = f"cfg2_planted_n{n}_r2_9"
    want = g[key][0] if key in g else oracle.count_i32(p["x"], p["y"], p["z"], 9)
    cc.set_tensor_cores(tc)
    try:
        got = gpu_count(cc, p["x"], p["y"], p["z"], 9)
        mode = cc.stream_mode()
    finally:
        cc.set_tensor_cores(True)
    assert mode == (cc.MODE_TENSOR if tc else cc.MODE_FP32_EXACT)
    assert got == want
    # the planted pairs alone: every pair among the planted objects collides
    k = len(synth.planted_positions(n))
    assert want >= k * (k - 1) // 2


def test_cfg3_full_size(cc):
    g = _golden()
    c = synth.cfg3()
    if "cfg3_n131072_f32" in g:
        want_c, want_s = g["cfg3_n131072_f32"]
    else:
        want_c, want_s = oracle.count_f32(c["x"], c["y"], c["z"], c["r"])
    assert gpu_count(cc, c["x"], c["y"], c["z"], 0, c["r"]) == want_c
    s, cnt = gpu_sum(cc, c["x"], c["y"], c["z"], 0, c["r"])
    assert cnt == want_c
    assert rel(s, want_s) <= SUM_RTOL


@pytest.mark.parametrize("n", [2, 3, 100, 385, 1023, 1024, 1025, 5000, 65537])
def test_straightforward_schedule_parity(cc, n):
    """The comparison kernel (every object against all later ones) counts the same pairs."""
    rng = np.random.default_rng(77 + n)
    x, y, z = (rng.integers(0, 20, n).astype(np.int32) for _ in range(3))
    t = dev(x, y, z)
    got = cc.count_pairs_straightforward(*t, r2=4)
    torch.cuda.synchronize()
    assert cc.as_u64(got) == oracle.count_i32(x, y, z, 4)
    xs, ys, zs, rs = synth.sphere_points(n, 5 + n, rmin=0.01, rmax=0.03)
    tf = dev(xs, ys, zs, rs)
    got = cc.count_pairs_straightforward(*tf[:3], r=tf[3])
    torch.cuda.synchronize()
    assert cc.as_u64(got) == oracle.count_f32(xs, ys, zs, rs)[0]
