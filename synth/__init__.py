"""Seeded synthetic inputs shared by the oracle-side tests, the GPU tests and bench.py.

This module holds only random-number generation and workload shapes. It contains none
of the counting method's arithmetic, so both the CPU oracle and the CUDA path can take
their inputs from here without sharing any part of the computation.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; constants as published by Vigna), used in counter mode:
draw k of stream `sid` under `seed` is mix(seed + (sid * 2**40 + k + 1) * GOLDEN).
Every transformation below uses integer arithmetic or IEEE basic operations only
(no libm calls), so the same seed gives the same bytes on x86-64 and on aarch64.

Workloads (the paper's GPU experiment draws random floating-point spheres, Section 5;
its CPU experiments draw random integer bead chains, Section 5):
  cfg1  N=4096 int32 points uniform in [0,64)^3, r2=16
  cfg2  N=262144 and 262145 int32 points uniform in [0,1024)^3, r2=9;
        same-cell variant on [0,256)^3 with r2=0
  cfg3  N=131072 FP32 spheres, centres uniform in [0,1)^3, radii in [0.001,0.004]
  cfg4  ~100k pruned sets from 64 Gaussian clusters in [0,4096)^3, sizes lognormal
        (mean ~40) clipped to [2,8192], int32, r2=25
  cfg5  a pool of resident sets with lognormal sizes in [16,65536] and a Poisson
        query stream over them
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 20190130


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def draws(seed: int, sid: int, count: int, start: int = 0) -> np.ndarray:
    """`count` uint64 draws of stream `sid`, counters start..start+count-1."""
    with np.errstate(over="ignore"):
        k = np.arange(start, start + count, dtype=np.uint64)
        base = np.uint64((int(sid) << 40) & 0xFFFFFFFFFFFFFFFF)
        ctr = base + k + np.uint64(1)
        z = np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF) + ctr * GOLDEN
        return _mix(z)


def uniform_bits(seed: int, sid: int, count: int, bits: int) -> np.ndarray:
    """Integers uniform in [0, 2**bits): the top `bits` bits of each draw."""
    assert 1 <= bits <= 31
    return (draws(seed, sid, count) >> np.uint64(64 - bits)).astype(np.int32)


def uniform_f32(seed: int, sid: int, count: int) -> np.ndarray:
    """FP32 values uniform in [0,1): (u >> 40) * 2**-24, exact in FP32."""
    u = draws(seed, sid, count) >> np.uint64(40)
    return (u.astype(np.float64) * (2.0 ** -24)).astype(np.float32)


def uniform_f64(seed: int, sid: int, count: int) -> np.ndarray:
    """FP64 values uniform in [0,1): (u >> 11) * 2**-53."""
    u = draws(seed, sid, count) >> np.uint64(11)
    return u.astype(np.float64) * (2.0 ** -53)


def gauss_fixed(seed: int, sid: int, count: int) -> np.ndarray:
    """Approximately standard-normal values as exact integers scaled by 2**32.

    Irwin-Hall: the sum of 12 independent 32-bit uniforms, minus 6. Returned as int64
    numerators over 2**32 so that callers can scale and floor in exact integer
    arithmetic (platform independent, unlike Box-Muller through libm).
    """
    u = draws(seed, sid, 12 * count) >> np.uint64(32)
    s = u.astype(np.int64).reshape(count, 12).sum(axis=1)
    return s - np.int64(6) * np.int64(1 << 32)


def _exp2_det(y: np.ndarray) -> np.ndarray:
    """2**y in FP64 with basic operations only (deterministic across platforms)."""
    y = np.asarray(y, dtype=np.float64)
    k = np.floor(y)
    f = y - k  # in [0,1)
    # 2**f = exp(f ln2) by a fixed 20-term Taylor series (|f ln2| < 0.7, error < 1e-16)
    t = f * 0.6931471805599453
    acc = np.ones_like(t)
    term = np.ones_like(t)
    for n in range(1, 21):
        term = term * t / float(n)
        acc = acc + term
    return np.ldexp(acc, k.astype(np.int64))


def lognormal_sizes(seed: int, sid: int, count: int, median: float, sigma: float,
                    lo: int, hi: int) -> np.ndarray:
    """Integer sizes round(median * exp(sigma * g)) clipped to [lo, hi]."""
    g = gauss_fixed(seed, sid, count).astype(np.float64) * (2.0 ** -32)
    log2e = 1.4426950408889634
    v = median * _exp2_det(sigma * g * log2e)
    n = np.floor(v + 0.5).astype(np.int64)
    return np.clip(n, lo, hi)


# --------------------------------------------------------------------------------------
# Workload builders
# --------------------------------------------------------------------------------------

def int_points(n: int, bits: int, seed: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """n int32 points uniform in [0, 2**bits)^3 (SoA)."""
    return (uniform_bits(seed, 1, n, bits), uniform_bits(seed, 2, n, bits),
            uniform_bits(seed, 3, n, bits))


def sphere_points(n: int, seed: int, rmin: float = 0.001, rmax: float = 0.004):
    """n FP32 spheres: centres uniform in [0,1)^3, radii uniform in [rmin, rmax]."""
    x = uniform_f32(seed, 1, n)
    y = uniform_f32(seed, 2, n)
    z = uniform_f32(seed, 3, n)
    r = (rmin + (rmax - rmin) * uniform_f64(seed, 4, n)).astype(np.float32)
    return x, y, z, r


def unit_spheres(n: int, box: float = 200.0, seed: int = SEED_BASE + 6):
    """n FP32 spheres of diameter 1 (radius 0.5), centres uniform in [0, box)^3: the
    shape of the paper's GPU experiment (random FP spheres of diameter 1, Section 5; the
    box size is not stated there)."""
    x = (uniform_f64(seed, 1, n) * box).astype(np.float32)
    y = (uniform_f64(seed, 2, n) * box).astype(np.float32)
    z = (uniform_f64(seed, 3, n) * box).astype(np.float32)
    r = np.full(n, 0.5, dtype=np.float32)
    return x, y, z, r


def cfg1():
    seed = SEED_BASE + 1
    x, y, z = int_points(4096, 6, seed)
    return dict(x=x, y=y, z=z, r2=16, name="single set N=4096 int32 [0,64)^3 r2=16")


def cfg2(n: int = 262144, same_cell: bool = False):
    seed = SEED_BASE + 2
    bits = 8 if same_cell else 10
    x, y, z = int_points(n, bits, seed + (100 if same_cell else 0))
    r2 = 0 if same_cell else 9
    box = 1 << bits
    return dict(x=x, y=y, z=z, r2=r2,
                name=f"single set N={n} int32 [0,{box})^3 r2={r2}")


def planted_positions(n: int) -> list[int]:
    """Positions at which cfg2_planted places coincident objects: the first and last
    objects, the middle of the set and its neighbours, and the objects around n/2 and
    (n-1)/2 (for the proposed algorithm of Section 4 these pairs sit at both ends of an
    object's window, across the wrap from the last object to the first, and on the even-N
    extra step)."""
    h = (n - 1) // 2
    pos = {0, 1, h - 1, h, h + 1, n // 2 - 1, n // 2, n // 2 + 1, n - 2, n - 1, n // 3}
    return sorted(p for p in pos if 0 <= p < n)


def cfg2_planted(n: int = 262145):
    """cfg2(n) with the objects at planted_positions(n) moved onto one lattice site, so
    that every pair among them collides (all at squared distance 0 <= r2 = 9)."""
    c = cfg2(n)
    x, y, z = c["x"].copy(), c["y"].copy(), c["z"].copy()
    pos = np.array(planted_positions(n), dtype=np.int64)
    site = (511, 17, 1000)
    x[pos], y[pos], z[pos] = site
    return dict(x=x, y=y, z=z, r2=9,
                name=f"single set N={n} int32 [0,1024)^3 r2=9 with {len(pos)} coincident objects planted")


def cfg3(n: int = 131072):
    seed = SEED_BASE + 3
    x, y, z, r = sphere_points(n, seed)
    return dict(x=x, y=y, z=z, r=r,
                name=f"single set N={n} FP32 spheres [0,1)^3 r in [0.001,0.004]")


def cfg4_sizes(num_sets: int = 100_000, total: int = 4_000_000, seed: int | None = None):
    """Set sizes: lognormal with mean ~40 (sigma 1.2) clipped to [2, 8192], rescaled so
    the sum is ~total, with one set of 4096 and one of 8192 always present."""
    seed = SEED_BASE + 4 if seed is None else seed
    sigma = 1.2
    mean = total / num_sets
    median = mean * float(_exp2_det(np.array([-sigma * sigma / 2 * 1.4426950408889634]))[0])
    n = lognormal_sizes(seed, 10, num_sets, median, sigma, 2, 8192)
    if num_sets >= 2:
        n[0] = 8192
        n[num_sets // 2] = 4096
    # rescale the bulk (excluding the forced two) so that the sum is close to `total`
    rest = n.sum() - 8192 - 4096
    want = total - 8192 - 4096
    if rest > 0 and want > 0:
        scale = want / rest
        m = np.floor(n.astype(np.float64) * scale + 0.5).astype(np.int64)
        m = np.clip(m, 2, 8192)
        m[0] = 8192
        m[num_sets // 2] = 4096
        n = m
    return n.astype(np.int64)


def cfg4(num_sets: int = 100_000, total: int = 4_000_000):
    """Batched workload: many pruned sets of int32 points around 64 cluster centres.

    Each set's points are Gaussian (sigma = 20) around one of 64 cluster centres drawn
    uniformly in [0,4096)^3 and clamped to [0,4096)^3. Returns SoA arrays of all points
    concatenated, int64 offsets[num_sets+1] and r2 = 25.
    """
    seed = SEED_BASE + 4
    sizes = cfg4_sizes(num_sets, total, seed)
    offsets = np.zeros(num_sets + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    ntot = int(offsets[-1])
    centres = np.stack([uniform_bits(seed, 20 + a, 64, 12) for a in range(3)], axis=1)
    which = (draws(seed, 30, num_sets) >> np.uint64(58)).astype(np.int64)  # 0..63
    set_of_point = np.repeat(np.arange(num_sets), sizes)
    sigma = 20
    coords = []
    for a in range(3):
        g = gauss_fixed(seed, 40 + a, ntot)
        # floor(sigma * g / 2**32) in exact integer arithmetic
        d = np.floor_divide(g * sigma, np.int64(1 << 32))
        c = centres[which[set_of_point], a].astype(np.int64) + d
        coords.append(np.clip(c, 0, 4095).astype(np.int32))
    return dict(x=coords[0], y=coords[1], z=coords[2], offsets=offsets, r2=25,
                name=f"batched {num_sets} sets, {ntot} int32 points, r2=25")


def cfg5_pool(num_sets: int = 2048, seed: int | None = None):
    """Serving pool: sizes lognormal (median 512, sigma 1.5) clipped to [16, 65536].

    Returns a list of dicts; even-indexed sets are int32 points in [0,1024)^3, odd ones
    FP32 spheres as in cfg3. Points of set k use streams derived from k.
    """
    seed = SEED_BASE + 5 if seed is None else seed
    sizes = lognormal_sizes(seed, 10, num_sets, 512.0, 1.5, 16, 65536)
    pool = []
    for k in range(num_sets):
        n = int(sizes[k])
        s = seed * 1000003 + k
        if k % 2 == 0:
            x, y, z = int_points(n, 10, s)
            pool.append(dict(kind="i32", x=x, y=y, z=z, n=n))
        else:
            x, y, z, r = sphere_points(n, s)
            pool.append(dict(kind="f32", x=x, y=y, z=z, r=r, n=n))
    return pool


def cfg5_queries(num_queries: int, num_sets: int, rate_per_s: float, seed: int | None = None):
    """Poisson query stream: arrival times (s), set ids, ops.

    op 0 = int count (r2 = 9) on an int set, op 1 = FP32 count and op 2 = FP32 sum on an
    FP32 set. Half of the queries are int counts, a quarter each FP32 count / sum.
    Exponential inter-arrival gaps come from -ln(u) computed by a fixed series
    (platform independent).
    """
    seed = SEED_BASE + 5 if seed is None else seed
    u = uniform_f64(seed, 50, num_queries)
    u = np.clip(u, 2.0 ** -53, 1.0)
    gaps = -_ln_det(u) / rate_per_s
    t = np.cumsum(gaps)
    kind = (draws(seed, 51, num_queries) >> np.uint64(62)).astype(np.int64)  # 0..3
    op = np.where(kind < 2, 0, kind - 1)  # 0,0,1,2
    pick = (draws(seed, 52, num_queries) >> np.uint64(33)).astype(np.int64)
    half = max(num_sets // 2, 1)
    sid = (pick % half) * 2 + np.where(op == 0, 0, 1)
    sid = np.minimum(sid, num_sets - 1)
    return dict(t=t, set_id=sid, op=op)


def _ln_det(u: np.ndarray) -> np.ndarray:
    """ln(u) for u in (0,1] with basic operations only: u = m * 2**e, m in [1,2),
    ln(m) = 2 atanh((m-1)/(m+1)) by a fixed odd series."""
    m, e = np.frexp(u)  # u = m * 2**e, m in [0.5,1)
    m = m * 2.0
    e = e - 1
    q = (m - 1.0) / (m + 1.0)
    q2 = q * q
    acc = np.zeros_like(q)
    for k in range(39, 0, -2):
        acc = acc * q2 + 1.0 / k
    return 2.0 * q * acc + e * 0.6931471805599453
