"""The exact integer screen of the tensor-core sphere form passes every pair that the FP32
predicate accepts (CPU, no GPU).

The device quantises each coordinate as X = floor((x - min) * S), S = 2046 / (largest
per-axis span), computed in FP64, and passes a pair when its integer squared distance
D^2 is at most r2q = ceil((2 rmax S (1 + 1e-6) + 1.7331)^2). These tests restate that
rule in numpy and check, on sets built to stress it, that no pair the FP32 predicate
accepts (the oracle's collide_f32, or the same operations in numpy float32) falls
outside the screen, and that the quantised coordinates stay in [0, 2046] (the range in
which the integer contraction is exact).
"""
import math

import numpy as np

import oracle
from tests.golden import make_near_ties as nt


def screen_params(x, y, z, r):
    lo = [float(np.min(a)) for a in (x, y, z)]
    span = max(float(np.max(a)) - l for a, l in zip((x, y, z), lo))
    S = 2046.0 / span if span > 0 else 1.0
    rmax = float(np.max(np.abs(r)))
    reach = 2.0 * rmax * S * (1.0 + 1e-6) + 1.7331
    return lo, S, math.ceil(reach * reach)


def quantise(a, lo, S):
    return np.floor((a.astype(np.float64) - lo) * S).astype(np.int64)


def predicate_f32(xi, yi, zi, ri, xj, yj, zj, rj):
    """The FP32 predicate, elementwise: numpy float32 arithmetic rounds every operation to
    nearest and never fuses, in the order written."""
    dx, dy, dz = xi - xj, yi - yj, zi - zj
    d2 = (dx * dx + dy * dy) + dz * dz
    s = ri + rj
    return d2 <= s * s


def check_set(x, y, z, r, pairs=None):
    x, y, z, r = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, y, z, r))
    lo, S, r2q = screen_params(x, y, z, r)
    X, Y, Z = quantise(x, lo[0], S), quantise(y, lo[1], S), quantise(z, lo[2], S)
    for Q in (X, Y, Z):
        assert Q.min() >= 0 and Q.max() <= 2046
    n = len(x)
    hits = 0
    if pairs is None:
        for i in range(n - 1):
            j = np.arange(i + 1, n)
            acc = predicate_f32(x[i], y[i], z[i], r[i], x[j], y[j], z[j], r[j])
            if not acc.any():
                continue
            jj = j[acc]
            D2 = (X[jj] - X[i]) ** 2 + (Y[jj] - Y[i]) ** 2 + (Z[jj] - Z[i]) ** 2
            assert (D2 <= r2q).all(), (i, jj[D2 > r2q][:5], r2q)
            hits += int(acc.sum())
    else:
        for i, j in pairs:
            if oracle.collide_f32((x[i], y[i], z[i], r[i]), (x[j], y[j], z[j], r[j])):
                D2 = (X[j] - X[i]) ** 2 + (Y[j] - Y[i]) ** 2 + (Z[j] - Z[i]) ** 2
                assert D2 <= r2q, (i, j, D2, r2q)
                hits += 1
    return hits, r2q


def test_numpy_predicate_matches_oracle():
    rng = np.random.default_rng(40)
    a = rng.random((2000, 4)).astype(np.float32) * np.float32([1, 1, 1, 0.05])
    b = (a + rng.normal(0, 0.03, a.shape)).astype(np.float32)
    b[:, 3] = np.abs(b[:, 3])
    got = predicate_f32(*(a[:, k] for k in range(4)), *(b[:, k] for k in range(4)))
    want = [oracle.collide_f32(a[k], b[k]) for k in range(len(a))]
    assert got.tolist() == [bool(w) for w in want]
    assert 0 < sum(want) < len(want)


def test_near_tie_fixture():
    """Pairs decided by the predicate's rounding: accepted ones are inside the screen."""
    pts = nt.load()
    pairs = [(k, k + 1) for k in range(0, len(pts), 2)]
    hits, _ = check_set(pts[:, 0], pts[:, 1], pts[:, 2], pts[:, 3], pairs)
    assert hits > 0


def test_touching_spheres_at_the_largest_radius():
    """Pairs at distance (r_i + r_j)(1 + k ulp) for the largest radii, along diagonals,
    in a set whose span makes 2 rmax S large (r2q near the admission limit)."""
    rng = np.random.default_rng(41)
    rmax = np.float32(0.0105)
    base = rng.random((600, 3)).astype(np.float32) * np.float32(0.9) + np.float32(0.05)
    direc = rng.normal(size=(600, 3))
    direc /= np.linalg.norm(direc, axis=1, keepdims=True)
    scale = (2.0 * float(rmax)) * (1.0 + rng.integers(-4, 5, 600) * 2.0 ** -23)
    other = (base + direc * scale[:, None]).astype(np.float32)
    pts = np.concatenate([base, other])
    r = np.full(len(pts), rmax, np.float32)
    pts[0] = 0.0
    pts[1] = 1.0
    pairs = [(k, k + 600) for k in range(600)]
    hits, r2q = check_set(pts[:, 0], pts[:, 1], pts[:, 2], r, pairs)
    assert hits > 100 and 1900 < r2q <= 2048


def test_random_sets_all_pairs():
    rng = np.random.default_rng(42)
    for n, lo_r, hi_r, box in ((3000, 0.002, 0.01, 1.0), (2500, 1e-23, 5e-23, 1e-20),
                               (2000, 0.3, 0.5, 100.0)):
        x, y, z = (rng.random(n, dtype=np.float32) * np.float32(box) for _ in range(3))
        r = (lo_r + (hi_r - lo_r) * rng.random(n)).astype(np.float32)
        hits, _ = check_set(x, y, z, r)
        assert hits == oracle.count_f32(x, y, z, r)[0]


def test_coincident_and_clustered():
    rng = np.random.default_rng(43)
    n = 1500
    x = np.full(n, 0.25, np.float32)
    r = np.full(n, 0.001, np.float32)
    hits, r2q = check_set(x, x.copy(), x.copy(), r)
    assert hits == n * (n - 1) // 2 and r2q == math.ceil((0.002 * (1 + 1e-6) + 1.7331) ** 2)
    x, y, z = (np.float32(0.5) + np.float32(0.01) * rng.random(n, dtype=np.float32) for _ in range(3))
    x[0], x[1] = np.float32(0.0), np.float32(1.0)
    r = (0.001 + 0.003 * rng.random(n)).astype(np.float32)
    hits, _ = check_set(x, y, z, r)
    assert hits == oracle.count_f32(x, y, z, r)[0]
