"""Pins for the CPU oracle: checks against facts fixed by the paper and by mathematics.

Each pin takes the oracle module (or a planted-mistake build of it loaded the same way)
and raises AssertionError when the oracle disagrees. None of them re-types the oracle's
loop: they use closed forms, combinatorial counts, the paper's worked example, its
propositions, Algorithms 1 and 2 as independent counters, symmetry, and brute force over
ordered pairs with a different structure (all N*N ordered pairs, then halved).

The paper is Saldanha and de Souza, arXiv 1901.11204.
"""
from __future__ import annotations

import itertools
import math
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---- helpers (no pair loop of the method) -----------------------------------------

def lattice_pairs_closed_form(L, r2):
    """Unordered pairs of distinct sites of an Lx*Ly*Lz lattice box with squared
    distance <= r2: half the sum over non-zero offsets d with |d|^2 <= r2 of
    prod_a max(L_a - |d_a|, 0) (each offset vector fits that many times)."""
    Lx, Ly, Lz = L
    m = int(math.isqrt(r2))
    total = 0
    for dx in range(-m, m + 1):
        for dy in range(-m, m + 1):
            for dz in range(-m, m + 1):
                if (dx, dy, dz) == (0, 0, 0) or dx * dx + dy * dy + dz * dz > r2:
                    continue
                total += (max(Lx - abs(dx), 0) * max(Ly - abs(dy), 0) * max(Lz - abs(dz), 0))
    assert total % 2 == 0
    return total // 2


def lattice_points(L, rng):
    Lx, Ly, Lz = L
    g = np.stack(np.meshgrid(np.arange(Lx), np.arange(Ly), np.arange(Lz), indexing="ij"), -1)
    p = g.reshape(-1, 3).astype(np.int32)
    p = p[rng.permutation(len(p))]
    return p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy()


def ordered_pairs_bruteforce_i32(x, y, z, r2):
    """All N*N ordered pairs through a distance matrix; drop the diagonal; halve."""
    P = np.stack([x, y, z], 1).astype(np.int64)
    D = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    hits = int((D <= r2).sum()) - len(x)
    assert hits % 2 == 0
    return hits // 2


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            out[k] = [int(t) for t in v]
    return out


# ---- pins: the proposed cyclic schedule (Section 4) ---------------------------------

def pin_fig1_worked_example(o):
    """Section 4, Figure 1: N=5, bead 1 reaches 2 and 3, is reached by 0 and 4; step
    (N+1)/2 = 3 would repeat an interaction."""
    g = read_golden("fig1_cyclic_n5.txt")
    n, bead = g["n"][0], g["bead"][0]
    pi, pj = o.cyclic_schedule(n)
    reaches = [int(j) for i, j in zip(pi, pj) if i == bead]
    reached_by = [int(i) for i, j in zip(pi, pj) if j == bead]
    assert reaches == g["reaches"], (reaches, g["reaches"])
    assert reached_by == g["reached_by"], (reached_by, g["reached_by"])
    # the step after the last one evaluates a pair already seen
    s = g["first_repeat_step"][0]
    assert s == (n + 1) // 2
    j3 = (g["reaches"][-1] + s) % n  # what bead reaches(3) would give for bead 3
    assert j3 == bead


def pin_cyclic_covers_every_pair_once(o):
    """Propositions 1 and 2 plus the even-N rule: for every N the schedule evaluates
    N(N-1)/2 pairs, all distinct, covering every unordered pair."""
    for n in list(range(0, 130)) + [255, 256, 257, 500, 501]:
        pi, pj = o.cyclic_schedule(n)
        assert len(pi) == n * (n - 1) // 2, (n, len(pi))
        if n < 2:
            continue
        assert np.all(pi != pj)
        key = np.minimum(pi, pj) * n + np.maximum(pi, pj)
        assert len(np.unique(key)) == len(key), n
        assert np.all((pj >= 0) & (pj < n))


def pin_cyclic_balance_and_depth(o):
    """Section 4: every object does (N-1)/2 evaluations; for even N the first half does
    one more, so the depth is (N-1)/2 for odd N and N/2 for even N."""
    for n in [2, 3, 4, 5, 6, 7, 8, 63, 64, 65, 1000, 1001]:
        pi, _ = o.cyclic_schedule(n)
        per_i = np.bincount(pi, minlength=n)
        for i in range(n):
            want = (n - 1) // 2 + (1 if (n % 2 == 0 and i < n // 2) else 0)
            assert per_i[i] == want == o.cyclic_work(n, i), (n, i, per_i[i], want)
        depth = per_i.max()
        assert depth == ((n - 1) // 2 if n % 2 else n // 2)


# ---- pins: integer collision counts --------------------------------------------------

def pin_all_identical(o):
    """Every pair collides when all points coincide: N(N-1)/2 (Proposition 1)."""
    for n in [0, 1, 2, 3, 4, 5, 64, 65, 257]:
        v = np.full(n, 7, dtype=np.int32)
        for r2 in [0, 9]:
            assert o.count_i32(v, v + 1, v - 3, r2) == n * (n - 1) // 2
            assert o.count_i32_cyclic(v, v + 1, v - 3, r2) == n * (n - 1) // 2


def pin_well_separated(o):
    """Points on a grid of spacing 4 never collide for r2 < 16 and the nearest
    neighbours appear exactly at r2 = 16."""
    rng = np.random.default_rng(1)
    x, y, z = lattice_points((5, 6, 7), rng)
    x, y, z = x * 4, y * 4, z * 4
    assert o.count_i32(x, y, z, 15) == 0
    assert o.count_i32(x, y, z, 16) == lattice_pairs_closed_form((5, 6, 7), 1)


def pin_line_closed_form(o):
    """Points at integer positions 0..N-1 on one axis (permuted): pairs with
    |i-j| <= k number sum_{m=1}^{min(k,N-1)} (N-m). Each axis separately."""
    rng = np.random.default_rng(2)
    for n in [1, 2, 7, 64, 65]:
        for axis in range(3):
            c = [np.full(n, 3, dtype=np.int32) for _ in range(3)]
            c[axis] = rng.permutation(n).astype(np.int32)
            for k in sorted({0, 1, 3, n // 2, n}):
                want = sum(n - m for m in range(1, min(k, n - 1) + 1))
                assert o.count_i32(*c, k * k) == want, (n, axis, k)
                assert o.count_i32_cyclic(*c, k * k) == want, (n, axis, k)
                # r2 just below k^2 loses exactly the pairs at distance k
                if k >= 1:
                    below = want - (n - k if k <= n - 1 else 0)
                    assert o.count_i32(*c, k * k - 1) == below, (n, axis, k)


def pin_lattice_closed_form(o):
    """All sites of a non-cubic box, permuted: the count for every r2 equals the
    combinatorial closed form (catches a dropped, doubled or swapped axis)."""
    rng = np.random.default_rng(3)
    for L in [(3, 4, 5), (6, 2, 7), (1, 9, 4)]:
        x, y, z = lattice_points(L, rng)
        for r2 in [0, 1, 2, 3, 4, 5, 6, 8, 9, 12, 17]:
            want = lattice_pairs_closed_form(L, r2)
            assert o.count_i32(x, y, z, r2) == want, (L, r2)
            assert o.count_i32_cyclic(x, y, z, r2) == want, (L, r2)
    # textbook forms for r2 = 1, 2, 3 on an L^3 cube
    Lc = 5
    x, y, z = lattice_points((Lc, Lc, Lc), rng)
    f1 = 3 * Lc * Lc * (Lc - 1)
    f2 = f1 + 6 * Lc * (Lc - 1) ** 2
    f3 = f2 + 4 * (Lc - 1) ** 3
    assert [o.count_i32(x, y, z, r) for r in (1, 2, 3)] == [f1, f2, f3]


def pin_bruteforce_small(o):
    """Random tiny inputs against all ordered pairs through a distance matrix."""
    rng = np.random.default_rng(4)
    for trial in range(60):
        n = int(rng.integers(0, 65))
        box = int(rng.choice([2, 4, 8, 16]))
        x, y, z = (rng.integers(-box, box, n).astype(np.int32) for _ in range(3))
        r2 = int(rng.integers(0, 3 * box * box))
        want = ordered_pairs_bruteforce_i32(x, y, z, r2)
        assert o.count_i32(x, y, z, r2) == want, (trial, n, r2)
        assert o.count_i32_cyclic(x, y, z, r2) == want, (trial, n, r2)


def pin_permutation_invariance(o):
    """The count does not depend on the order of the objects (both parities)."""
    rng = np.random.default_rng(5)
    for n in [300, 301]:
        x, y, z = (rng.integers(0, 12, n).astype(np.int32) for _ in range(3))
        base = o.count_i32(x, y, z, 4)
        for _ in range(3):
            p = rng.permutation(n)
            assert o.count_i32(x[p], y[p], z[p], 4) == base
            assert o.count_i32_cyclic(x[p], y[p], z[p], 4) == base
        assert o.count_i32(x[::-1], y[::-1], z[::-1], 4) == base


def pin_same_site_algorithm1(o):
    """Algorithm 1 (Section 3) counts same-site collisions in O(N): it must equal the
    r2 = 0 pair count and sum_k k(k-1)/2 over the site histogram."""
    rng = np.random.default_rng(6)
    for n, box in [(0, 4), (1, 4), (500, 4), (2001, 6), (3000, 16)]:
        x, y, z = (rng.integers(0, box, n).astype(np.int32) for _ in range(3))
        if n:
            _, k = np.unique(np.stack([x, y, z], 1), axis=0, return_counts=True)
            hist = int((k * (k - 1) // 2).sum())
        else:
            hist = 0
        assert o.count_colls(x, y, z) == hist
        assert o.count_i32(x, y, z, 0) == hist
        assert o.count_i32_cyclic(x, y, z, 0) == hist


def pin_contacts_algorithm2(o):
    """Algorithm 2 (Section 3) counts pairs on face-adjacent sites: it equals the pairs
    at squared distance exactly 1, i.e. count(r2=1) - count(r2=0)."""
    rng = np.random.default_rng(7)
    for n, box in [(400, 5), (1500, 9), (64, 3)]:
        x, y, z = (rng.integers(-box, box, n).astype(np.int32) for _ in range(3))
        assert o.count_contacts(x, y, z) == o.count_i32(x, y, z, 1) - o.count_i32(x, y, z, 0)
    # a random bead chain (Section 5's CPU workload): unit steps in 6 directions
    steps = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    ch = np.cumsum(steps[rng.integers(0, 6, 200)], axis=0).astype(np.int32)
    x, y, z = ch[:, 0].copy(), ch[:, 1].copy(), ch[:, 2].copy()
    assert o.count_contacts(x, y, z) == o.count_i32(x, y, z, 1) - o.count_i32(x, y, z, 0)
    assert o.count_colls(x, y, z) == o.count_i32(x, y, z, 0)


def pin_sets(o):
    """Per-set counts equal the single-set count of every slice; empty and one-point
    sets give 0."""
    rng = np.random.default_rng(8)
    sizes = np.array([0, 1, 2, 3, 17, 64, 65, 0, 130])
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    n = int(off[-1])
    x, y, z = (rng.integers(0, 6, n).astype(np.int32) for _ in range(3))
    got = o.count_i32_sets(x, y, z, off, 2)
    for k in range(len(sizes)):
        a, b = off[k], off[k + 1]
        assert int(got[k]) == ordered_pairs_bruteforce_i32(x[a:b], y[a:b], z[a:b], 2), k
    xf, yf, zf = x.astype(np.float32), y.astype(np.float32), z.astype(np.float32)
    rf = np.full(n, 0.75, dtype=np.float32)  # s = 1.5, s^2 = 2.25: same pairs as r2 = 2
    cnt, _ = o.count_f32_sets(xf, yf, zf, rf, off)
    assert np.array_equal(cnt, got)


def pin_f32_sets_sums(o):
    """Per-set FP32 counts and FP64 sums. (1) Every set is a permuted line of
    unit-spaced spheres of radius 1.5 along its own axis: pairs collide iff |i-j| <= 3,
    so set k of n objects has count sum_{m<=3} (n-m) and sum sum_{m<=3} (n-m)/m (the
    standard algorithm of Section 4 applied to each set alone; Fractions give the exact
    value). (2) On random sets each per-set sum equals the brute-force sum over all
    ordered pairs of that slice (exact-rational predicate, math.fsum, halved)."""
    rng = np.random.default_rng(15)
    sizes = [0, 1, 2, 3, 4, 7, 50, 0, 101, 5]
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    cols = [[], [], []]
    for k, n in enumerate(sizes):
        axis = k % 3
        for a in range(3):
            cols[a].append(rng.permutation(n).astype(np.float32) if a == axis
                           else np.full(n, 0.25 + k, dtype=np.float32))
    x, y, z = (np.concatenate(c) if c else np.zeros(0, np.float32) for c in cols)
    r = np.full(len(x), 1.5, dtype=np.float32)
    cnt, sm = o.count_f32_sets(x, y, z, r, off)
    for k, n in enumerate(sizes):
        want = sum(n - m for m in range(1, min(3, n - 1) + 1))
        wsum = sum(Fraction(n - m, m) for m in range(1, min(3, n - 1) + 1))
        assert int(cnt[k]) == want, (k, n, int(cnt[k]), want)
        assert abs(sm[k] - float(wsum)) <= 1e-12 * max(1.0, float(wsum)), (k, n, sm[k], wsum)
    # random small sphere sets against all ordered pairs of each slice
    sizes = [int(v) for v in rng.integers(0, 24, 6)]
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    m = int(off[-1])
    x, y, z = (rng.random(m).astype(np.float32) * np.float32(0.04) for _ in range(3))
    r = (0.002 + 0.01 * rng.random(m)).astype(np.float32)
    cnt, sm = o.count_f32_sets(x, y, z, r, off)
    for k in range(len(sizes)):
        a, b = int(off[k]), int(off[k + 1])
        terms = []
        for i, j in itertools.permutations(range(a, b), 2):
            if _spec_pred_exact((x[i], y[i], z[i], r[i]), (x[j], y[j], z[j], r[j])):
                d = math.sqrt(sum((float(p[i]) - float(p[j])) ** 2 for p in (x, y, z)))
                terms.append(1.0 / max(d, 1e-6))
        assert len(terms) % 2 == 0
        assert int(cnt[k]) == len(terms) // 2, (k, int(cnt[k]), len(terms))
        want = math.fsum(terms) / 2
        assert abs(sm[k] - want) <= 1e-12 * max(1.0, want), (k, sm[k], want)


# ---- pins: FP32 spheres ---------------------------------------------------------------

def pin_f32_line_closed_form(o):
    """Unit-spaced spheres of radius 1.5 on a line collide iff |i-j| <= 3 (s^2 = 9 is
    exact, touching counts): count = sum_{m<=3} (N-m), sum = sum_{m<=3} (N-m)/m."""
    rng = np.random.default_rng(9)
    for n in [1, 2, 3, 4, 5, 100, 101]:
        for axis in range(3):
            c = [np.full(n, 0.25, dtype=np.float32) for _ in range(3)]
            c[axis] = rng.permutation(n).astype(np.float32)
            r = np.full(n, 1.5, dtype=np.float32)
            cnt, sm = o.count_f32(*c, r)
            want = sum(n - m for m in range(1, min(3, n - 1) + 1))
            wsum = sum(Fraction(n - m, m) for m in range(1, min(3, n - 1) + 1))
            assert cnt == want, (n, axis, cnt, want)
            assert abs(sm - float(wsum)) <= 1e-12 * max(1.0, float(wsum)), (sm, wsum)


def pin_f32_two_radii(o):
    """Alternating radii 1 (even i) and 2 (odd i) at unit spacing: pairs at distance m
    collide iff m <= ri + rj; counted combinatorially (catches ri/rj mix-ups)."""
    for n in [2, 9, 10, 31]:
        x = np.arange(n, dtype=np.float32)
        zero = np.zeros(n, dtype=np.float32)
        r = np.where(np.arange(n) % 2 == 0, 1.0, 2.0).astype(np.float32)
        want = 0
        for i in range(n):
            for m in range(1, 5):
                j = i + m
                if j < n and m <= (1 if i % 2 == 0 else 2) + (1 if j % 2 == 0 else 2):
                    want += 1
        cnt, _ = o.count_f32(x, zero, zero, r)
        assert cnt == want, (n, cnt, want)
        cnt2, _ = o.count_f32(zero, x, zero, r)
        assert cnt2 == want


def pin_f32_ties_and_nan(o):
    """Touching spheres collide (<=), one ulp further they do not, NaN never collides,
    coincident centres give the 1/1e-6 term."""
    a = (0.0, 0.0, 0.0, 1.5)
    b = (3.0, 0.0, 0.0, 1.5)
    assert o.collide_f32(a, b) and o.collide_f32(b, a)
    b2 = (float(np.nextafter(np.float32(3.0), np.float32(4.0))), 0.0, 0.0, 1.5)
    assert not o.collide_f32(a, b2) and not o.collide_f32(b2, a)
    nan = float("nan")
    assert not o.collide_f32((nan, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0))
    assert not o.collide_f32((0.0, 0.0, 0.0, nan), (0.0, 0.0, 0.0, 1.0))
    x = np.array([0.5, 0.5, 0.75], dtype=np.float32)
    y = np.zeros(3, dtype=np.float32)
    r = np.array([0.01, 0.01, 0.001], dtype=np.float32)
    cnt, sm = o.count_f32(x, y, y, r)
    assert cnt == 1 and sm == 1e6


def _f32_round_exact(v: Fraction) -> float:
    """Round a rational to the nearest FP32 (ties to even), exactly."""
    if v == 0:
        return 0.0
    sign = -1 if v < 0 else 1
    a = abs(v)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)
    q = a / (Fraction(2) ** (e - 23))
    fl = q.numerator // q.denominator
    rem = q - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return sign * float(Fraction(fl) * Fraction(2) ** (e - 23))


def _spec_pred_exact(a, b):
    """The FP32 predicate evaluated with exact rational arithmetic and an explicit
    round-to-FP32 after every operation (independent of any float unit)."""
    F = Fraction
    rd = _f32_round_exact
    a = [float(v) for v in a]
    b = [float(v) for v in b]
    dx = rd(F(a[0]) - F(b[0]))
    dy = rd(F(a[1]) - F(b[1]))
    dz = rd(F(a[2]) - F(b[2]))
    d2 = rd(F(rd(F(rd(F(dx) * F(dx))) + F(rd(F(dy) * F(dy))))) + F(rd(F(dz) * F(dz))))
    s = rd(F(a[3]) + F(b[3]))
    s2 = rd(F(s) * F(s))
    return d2 <= s2


def pin_f32_rounding_near_ties(o):
    """Near-tie pairs where FP32 rounding after every step and exact real arithmetic
    disagree: the oracle must follow the FP32 rounding (checked with exact rationals
    rounded step by step), in both argument orders."""
    rng = np.random.default_rng(10)
    found = 0
    tries = 0
    while found < 40 and tries < 400000:
        tries += 1
        a = rng.random(4).astype(np.float32)
        a[3] = np.float32(0.002 + 0.002 * rng.random())
        direction = rng.standard_normal(3)
        direction /= np.linalg.norm(direction)
        rb = np.float32(0.001 + 0.003 * rng.random())
        dist = float(a[3]) + float(rb)
        b = np.empty(4, dtype=np.float32)
        b[:3] = (a[:3].astype(np.float64) + direction * dist).astype(np.float32)
        b[3] = rb
        # exact real-number decision on the FP32 inputs
        F = Fraction
        d2r = sum((F(float(a[k])) - F(float(b[k]))) ** 2 for k in range(3))
        s2r = (F(float(a[3])) + F(float(b[3]))) ** 2
        exact = d2r <= s2r
        spec = _spec_pred_exact([float(v) for v in a], [float(v) for v in b])
        if exact == spec:
            continue
        found += 1
        assert o.collide_f32(a, b) == spec, (a, b)
        assert o.collide_f32(b, a) == spec, (a, b)
    assert found >= 10, found


def pin_f32_symmetry(o):
    """The predicate is symmetric in its arguments on random pairs, so the proposed
    algorithm may evaluate a pair as (i, j) or (j, i)."""
    rng = np.random.default_rng(11)
    for _ in range(3000):
        a = rng.random(4).astype(np.float32) * np.float32(0.01)
        b = rng.random(4).astype(np.float32) * np.float32(0.01)
        assert o.collide_f32(a, b) == o.collide_f32(b, a)


def pin_f32_sum_bruteforce(o):
    """Random small sphere sets: count and FP64 sum against all ordered pairs with the
    exact-rational predicate and math.fsum of the terms, halved."""
    rng = np.random.default_rng(12)
    for trial in range(6):
        n = int(rng.integers(2, 40))
        x, y, z = (rng.random(n).astype(np.float32) * np.float32(0.05) for _ in range(3))
        r = (0.001 + 0.01 * rng.random(n)).astype(np.float32)
        terms = []
        cnt = 0
        for i, j in itertools.permutations(range(n), 2):
            if _spec_pred_exact((x[i], y[i], z[i], r[i]), (x[j], y[j], z[j], r[j])):
                cnt += 1
                d = math.sqrt(sum((float(p[i]) - float(p[j])) ** 2 for p in (x, y, z)))
                terms.append(1.0 / max(d, 1e-6))
        assert cnt % 2 == 0
        c, s = o.count_f32(x, y, z, r)
        assert c == cnt // 2, (trial, c, cnt)
        want = math.fsum(terms) / 2
        assert abs(s - want) <= 1e-12 * max(1.0, abs(want)), (s, want)


def pin_i32_sum_lattice(o):
    """All sites of a non-cubic box: each offset d (0 < |d|^2 <= r2) occurs
    prod_a (L_a - |d_a|) times as an ordered pair, so the count is half the sum of those
    multiplicities and the sum half the sum of multiplicity / |d|."""
    rng = np.random.default_rng(13)
    for L in [(5, 3, 4), (2, 7, 3)]:
        x, y, z = lattice_points(L, rng)
        for r2 in [1, 2, 5, 9]:
            m = math.isqrt(r2)
            cnt, terms = 0, []
            for d in itertools.product(range(-m, m + 1), repeat=3):
                d2 = sum(v * v for v in d)
                if d2 == 0 or d2 > r2:
                    continue
                mult = math.prod(max(L[a] - abs(d[a]), 0) for a in range(3))
                cnt += mult
                terms.append(mult / math.sqrt(d2))
            c, s = o.sum_i32(x, y, z, r2)
            assert c == cnt // 2 == o.count_i32(x, y, z, r2), (L, r2)
            want = math.fsum(terms) / 2
            assert abs(s - want) <= 1e-12 * want, (L, r2, s, want)


def pin_i32_sum_bruteforce(o):
    """Random small integer sets (with coincident points: each such pair adds 1e6)
    against all ordered pairs and math.fsum of the terms, halved."""
    rng = np.random.default_rng(14)
    for trial in range(8):
        n = int(rng.integers(2, 50))
        box = int(rng.choice([2, 3, 6]))
        x, y, z = (rng.integers(0, box, n).astype(np.int32) for _ in range(3))
        r2 = int(rng.integers(0, 3 * box * box))
        terms = []
        for i, j in itertools.permutations(range(n), 2):
            d2 = int(x[i] - x[j]) ** 2 + int(y[i] - y[j]) ** 2 + int(z[i] - z[j]) ** 2
            if d2 <= r2:
                terms.append(1.0 / max(math.sqrt(d2), 1e-6))
        c, s = o.sum_i32(x, y, z, r2)
        assert c == len(terms) // 2, (trial, c, len(terms))
        want = math.fsum(terms) / 2
        assert abs(s - want) <= 1e-12 * max(1.0, want), (trial, s, want)


ALL_PINS = [
    pin_fig1_worked_example,
    pin_cyclic_covers_every_pair_once,
    pin_cyclic_balance_and_depth,
    pin_all_identical,
    pin_well_separated,
    pin_line_closed_form,
    pin_lattice_closed_form,
    pin_bruteforce_small,
    pin_permutation_invariance,
    pin_same_site_algorithm1,
    pin_contacts_algorithm2,
    pin_sets,
    pin_f32_sets_sums,
    pin_f32_line_closed_form,
    pin_f32_two_radii,
    pin_f32_ties_and_nan,
    pin_f32_rounding_near_ties,
    pin_f32_symmetry,
    pin_f32_sum_bruteforce,
    pin_i32_sum_lattice,
    pin_i32_sum_bruteforce,
]
