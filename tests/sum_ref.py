"""FP64 reference for the interaction sum over integer points (test infrastructure).

The sum runs over unordered pairs whose exact integer squared distance d^2 is at most
r2, each pair adding 1/max(d, 1e-6) (d = sqrt(d^2); two coincident points add 1e6).
This is the plain definition, evaluated in FP64 by brute force over the pairs whose
x-distance can admit a hit (points sorted by x, so each point meets only the window of
later points within floor(sqrt(r2)) in x). Pinned against an all-pairs loop and the
lattice closed form in test_sum_ref.py.
"""
from __future__ import annotations

import numpy as np


def pair_sum_ref(x, y, z, r2: int) -> tuple[float, int]:
    """(sum, count) over unordered pairs with d^2 <= r2."""
    P = np.stack([np.asarray(x), np.asarray(y), np.asarray(z)], 1).astype(np.int64)
    P = P[np.argsort(P[:, 0], kind="stable")]
    reach = int(np.floor(np.sqrt(r2)))
    hi = np.searchsorted(P[:, 0], P[:, 0] + reach, side="right")
    tot, cnt = 0.0, 0
    for i in range(len(P) - 1):
        d2 = ((P[i + 1:hi[i]] - P[i]) ** 2).sum(1)
        hit = d2[d2 <= r2].astype(np.float64)
        cnt += hit.size
        tot += float((1.0 / np.maximum(np.sqrt(hit), 1e-6)).sum())
    return tot, cnt
