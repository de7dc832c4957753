"""FP32 spheres on the tensor cores (exact integer screen, then the FP32 predicate) against
the CPU oracle, through the C ABI.

The device admits the screened form when every coordinate and radius is finite and the
largest 2|r| is small against the largest coordinate span; then counts must equal the
oracle's bit for bit (the predicate's specified rounding included) and sums agree to
1e-5. The tests cover ragged sizes, both parities, the near-tie fixture embedded in a
large set, coincident points (every pair screened), coordinates whose squared distances
underflow, the fall-backs to the FP32-pipe kernel, and equality with that kernel.
"""
import numpy as np
import pytest

import oracle
from tests.golden import make_near_ties as nt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TC_MIN_N = 8192
SUM_RTOL = 1e-5


@pytest.fixture(scope="module")
def cc():
    import paper_1901_11204_gb300 as cc
    cc.build()
    cc.lib()
    return cc


def spheres(rng, n, lo=0.002, hi=0.01, box=1.0):
    x, y, z = (rng.random(n, dtype=np.float32) * np.float32(box) for _ in range(3))
    r = (lo + (hi - lo) * rng.random(n)).astype(np.float32)
    return x, y, z, r


def run(cc, x, y, z, r, tensor=True):
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, y, z, r)]
    cc.set_tensor_cores(tensor)
    try:
        c1 = cc.count_pairs(t[0], t[1], t[2], r=t[3])
        torch.cuda.synchronize()
        m1 = cc.stream_mode()
        s, c2 = cc.interaction_sum(t[0], t[1], t[2], r=t[3])
        torch.cuda.synchronize()
        m2 = cc.stream_mode()
    finally:
        cc.set_tensor_cores(True)
    assert m1 == m2
    assert cc.as_u64(c1) == cc.as_u64(c2)
    return cc.as_u64(c1), float(s.item()), m1


def check(cc, x, y, z, r, want_mode):
    c, s, mode = run(cc, x, y, z, r)
    assert mode == want_mode, mode
    want_c, want_s = oracle.count_f32(x, y, z, r)
    assert c == want_c
    assert abs(s - want_s) <= SUM_RTOL * max(abs(want_s), 1e-30)
    return c, s


@pytest.mark.parametrize("n", [8192, 8193, 16384, 16385, 20001, 33026])
def test_counts_and_sums_on_tensor_cores(cc, n):
    rng = np.random.default_rng(300 + n)
    x, y, z, r = spheres(rng, n)
    c, s = check(cc, x, y, z, r, cc.MODE_TENSOR_SPHERES)
    assert c > 100
    c2, s2, mode2 = run(cc, x, y, z, r, tensor=False)
    assert mode2 == cc.MODE_FP32_SPHERES and c2 == c
    assert abs(s - s2) <= SUM_RTOL * s


def test_near_tie_fixture_in_a_large_set(cc):
    """The 240 near-tie pairs (each decided by the predicate's rounding) among 20,000
    other spheres: the screen passes them and the FP32 predicate decides them."""
    pts = nt.load()
    rng = np.random.default_rng(301)
    fx, fy, fz, fr = spheres(rng, 20000, 0.001, 0.003)
    fz = (np.float32(0.6) + np.float32(0.4) * fz).astype(np.float32)   # apart from the fixture (z < 0.48)
    x = np.concatenate([pts[:, 0], fx]); y = np.concatenate([pts[:, 1], fy])
    z = np.concatenate([pts[:, 2], fz]); r = np.concatenate([pts[:, 3], fr])
    p = rng.permutation(len(x))
    x, y, z, r = (np.ascontiguousarray(a[p]) for a in (x, y, z, r))
    check(cc, x, y, z, r, cc.MODE_TENSOR_SPHERES)


def test_coincident_points(cc):
    """Span 0: every pair is screened and collides."""
    n = 16400
    x = np.full(n, 0.25, np.float32)
    r = np.full(n, 0.001, np.float32)
    c, s, mode = run(cc, x, x.copy(), x.copy(), r)
    assert mode == cc.MODE_TENSOR_SPHERES
    assert c == n * (n - 1) // 2
    want = c / np.float32(1e-6)
    assert abs(s - want) <= SUM_RTOL * want


def test_underflowing_distances(cc):
    """Coordinates near 1e-20: squared distances fall in or below the subnormal range,
    where the FP32 rounding (not the real distance) decides."""
    rng = np.random.default_rng(302)
    n = 20000
    x, y, z, r = spheres(rng, n, 1e-23, 5e-23, box=1e-20)
    check(cc, x, y, z, r, cc.MODE_TENSOR_SPHERES)


def test_fall_backs(cc):
    rng = np.random.default_rng(303)
    # radii too large against the span: the screen would pass too many pairs
    x, y, z, r = spheres(rng, 20000, 0.01, 0.03)
    check(cc, x, y, z, r, cc.MODE_FP32_SPHERES)
    # a NaN coordinate or an infinite radius: the FP32-pipe kernel
    x, y, z, r = spheres(rng, 20000)
    x[17] = np.nan
    check(cc, x, y, z, r, cc.MODE_FP32_SPHERES)
    x, y, z, r = spheres(rng, 20000)
    r[5] = np.inf
    c, _, mode = run(cc, x, y, z, r)
    assert mode == cc.MODE_FP32_SPHERES and c == oracle.count_f32(x, y, z, r)[0]
    # below the size threshold
    x, y, z, r = spheres(rng, TC_MIN_N - 1)
    check(cc, x, y, z, r, cc.MODE_FP32_SPHERES)


def test_admission_boundary(cc):
    """Largest span exactly 1 (S = 2046): the largest radius 0.010635799 gives r2q = 2048
    (admitted), the next float 0.0106358 gives 2049 (FP32 pipe); exact either way."""
    rng = np.random.default_rng(305)
    n = 12000
    x, y, z, r = spheres(rng, n, 0.002, 0.005)
    x[0], y[0], z[0] = 0.0, 0.0, 0.0
    x[1] = 1.0
    for rmax, want in ((np.float32(0.010635799), cc.MODE_TENSOR_SPHERES),
                       (np.float32(0.0106358), cc.MODE_FP32_SPHERES)):
        r2 = r.copy()
        r2[7] = rmax
        check(cc, x, y, z, r2, want)


def test_clustered_points(cc):
    """Half the points in a small cluster: many screened pairs, exact all the same."""
    rng = np.random.default_rng(304)
    x, y, z, r = spheres(rng, 24000, 0.001, 0.004)
    k = 12000
    for a in (x, y, z):
        a[:k] = (np.float32(0.5) + np.float32(0.02) * rng.random(k, dtype=np.float32)).astype(np.float32)
    check(cc, x, y, z, r, cc.MODE_TENSOR_SPHERES)
