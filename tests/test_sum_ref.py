"""Pins for the FP64 interaction-sum reference used by the GPU sum tests."""
import math

import numpy as np

import oracle
from tests.sum_ref import pair_sum_ref


def all_pairs(x, y, z, r2):
    """Every ordered pair (i, j), i != j, then halved: a different loop structure."""
    P = np.stack([x, y, z], 1).astype(np.int64)
    d2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(2)
    off = ~np.eye(len(P), dtype=bool)
    hit = d2[(d2 <= r2) & off].astype(np.float64)
    return float((1.0 / np.maximum(np.sqrt(hit), 1e-6)).sum()) / 2, hit.size // 2


def test_against_all_ordered_pairs():
    rng = np.random.default_rng(5)
    for n, box, r2 in ((300, 12, 9), (257, 40, 400), (200, 3, 0), (150, 8, 2000)):
        x, y, z = (rng.integers(0, box, n).astype(np.int32) for _ in range(3))
        s, c = pair_sum_ref(x, y, z, r2)
        s2, c2 = all_pairs(x, y, z, r2)
        assert c == c2 == oracle.count_i32(x, y, z, r2)
        assert math.isclose(s, s2, rel_tol=1e-12)


def test_lattice_closed_form():
    """An Lx*Ly*Lz lattice: each non-zero offset d with |d|^2 <= r2 occurs
    prod_a (L_a - |d_a|) times as an ordered pair; unordered sum = half of
    sum_d mult(d) / |d|."""
    L = (7, 5, 4)
    r2 = 6
    g = np.stack(np.meshgrid(*[np.arange(k) for k in L], indexing="ij"), -1).reshape(-1, 3)
    want_s, want_c = 0.0, 0
    m = math.isqrt(r2)
    for dx in range(-m, m + 1):
        for dy in range(-m, m + 1):
            for dz in range(-m, m + 1):
                d2 = dx * dx + dy * dy + dz * dz
                if d2 == 0 or d2 > r2:
                    continue
                mult = max(L[0] - abs(dx), 0) * max(L[1] - abs(dy), 0) * max(L[2] - abs(dz), 0)
                want_c += mult
                want_s += mult / math.sqrt(d2)
    s, c = pair_sum_ref(g[:, 0], g[:, 1], g[:, 2], r2)
    assert c == want_c // 2
    assert math.isclose(s, want_s / 2, rel_tol=1e-12)


def test_coincident_points():
    x = np.zeros(5, np.int32)
    s, c = pair_sum_ref(x, x, x, 0)
    assert c == 10 and math.isclose(s, 10 * 1e6, rel_tol=1e-12)
