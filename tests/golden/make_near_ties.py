"""Writes tests/golden/f32_near_ties.txt: FP32 sphere pairs on the edge of collision.

Each line holds two spheres (x, y, z, r as FP32 bit patterns in hex) chosen so that the
specified evaluation (every operation rounded to FP32, (dx*dx + dy*dy) + dz*dz, no fused
multiply-add) decides differently from at least one plausible deviation: a fused
multiply-add in either sum, or exact real arithmetic. Pair k sits in its own cell of an
8x8x8 grid over [0,1)^3, so spheres of different pairs never touch. The file holds
inputs only; expected counts are computed by the oracle at test time.

Run from the repository root:  python tests/golden/make_near_ties.py
"""
import os
import sys
from fractions import Fraction as F

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from tests.pins import _f32_round_exact as rd  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "f32_near_ties.txt")


def _sq(v):
    return rd(F(v) * F(v))


def decisions(a, b):
    dx = rd(F(a[0]) - F(b[0]))
    dy = rd(F(a[1]) - F(b[1]))
    dz = rd(F(a[2]) - F(b[2]))
    s = rd(F(a[3]) + F(b[3]))
    s2 = rd(F(s) * F(s))
    spec = rd(F(rd(F(_sq(dx)) + F(_sq(dy)))) + F(_sq(dz))) <= s2
    f1 = rd(F(dz) * F(dz) + F(rd(F(dx) * F(dx) + F(_sq(dy))))) <= s2
    f2 = rd(F(dz) * F(dz) + F(rd(F(dy) * F(dy) + F(_sq(dx))))) <= s2
    f3 = rd(F(rd(F(_sq(dx)) + F(_sq(dy)))) + F(dz) * F(dz)) <= s2
    exact = (F(a[0]) - F(b[0])) ** 2 + (F(a[1]) - F(b[1])) ** 2 + (F(a[2]) - F(b[2])) ** 2 \
        <= (F(a[3]) + F(b[3])) ** 2
    return spec, (f1, f2, f3, exact)


def main(count=240, seed=20190130):
    rng = np.random.default_rng(seed)
    rows = []
    cell = 0
    while len(rows) < count:
        cx, cy, cz = cell % 8, (cell // 8) % 8, (cell // 64) % 8
        a = np.empty(4, dtype=np.float32)
        a[:3] = ((np.array([cx, cy, cz]) + 0.2 + 0.6 * rng.random(3)) / 8.0).astype(np.float32)
        a[3] = np.float32(0.001 + 0.003 * rng.random())
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        rb = np.float32(0.001 + 0.003 * rng.random())
        b = np.empty(4, dtype=np.float32)
        b[:3] = (a[:3].astype(np.float64) + d * (float(a[3]) + float(rb))).astype(np.float32)
        b[3] = rb
        af, bf = [float(v) for v in a], [float(v) for v in b]
        spec, others = decisions(af, bf)
        if any(o != spec for o in others):
            rows.append(np.concatenate([a, b]).view(np.uint32))
            cell += 1
            if cell >= 512:
                raise RuntimeError("more pairs than grid cells")
    with open(OUT, "w") as f:
        f.write("# FP32 near-tie sphere pairs (hex bit patterns): ax ay az ar bx by bz br\n")
        f.write("# written by tests/golden/make_near_ties.py; inputs only\n")
        for r in rows:
            f.write(" ".join(f"{int(v):08x}" for v in r) + "\n")
    print(f"wrote {len(rows)} pairs to {OUT}")


def load(path=OUT):
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    arr = np.array([[int(t, 16) for t in r] for r in rows], dtype=np.uint32).view(np.float32)
    a, b = arr[:, :4], arr[:, 4:]
    pts = np.empty((2 * len(arr), 4), dtype=np.float32)
    pts[0::2] = a
    pts[1::2] = b
    return pts


if __name__ == "__main__":
    main()
