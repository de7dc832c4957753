"""The admission bound of the tensor-core form, checked by brute force on the CPU.

The kernel writes d^2 - r2e - 1 as eight TF32 products
    a_i = [-2x_i, -2y_i, -2z_i, 1, 1, cA*2^22, cB*2^11, cC]
    b_j = [ x_j,   y_j,   z_j, nH*2^11, nL, 1, 1, 1]
(centred coordinates, n_j = |p_j|^2 = nH*2^11 + nL, c_i = n_i - r2e - 1 in balanced
base-2^11 digits) and admits a set only when 9m^2 + max(r2e + 1, 3m^2) + 2^22 + 2^11
< 2^24. These tests restate the digit split independently and check, over the extreme
coordinates of admitted (m, r2e), that every operand is exact in TF32 (at most 11
significant bits), that the digits reconstruct c_i, that the eight products sum to
d^2 - r2e - 1, and that the sum of their absolute values stays below 2^24 -- the
condition under which every partial sum, in any order, is an exact FP32 integer.
"""
import itertools

import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def admitted(m, r2e):
    c = max(r2e + 1, 3 * m * m)
    return 9 * m * m + c + (1 << 22) + 2048 < (1 << 24)


def balanced_digits(c):
    """c = cA*2^22 + cB*2^11 + cC with cB, cC in [-1024, 1023]."""
    cC = ((c + 1024) % 2048) - 1024
    c1 = (c - cC) // 2048
    cB = ((c1 + 1024) % 2048) - 1024
    cA = (c1 - cB) // 2048
    return cA, cB, cC


def sig_bits(v):
    """Significant bits of an integer (0 for 0): odd part's bit length."""
    v = abs(int(v))
    if v == 0:
        return 0
    while v % 2 == 0:
        v //= 2
    return v.bit_length()


def operands(pi, pj, r2e):
    ni = sum(t * t for t in pi)
    nj = sum(t * t for t in pj)
    cA, cB, cC = balanced_digits(ni - r2e - 1)
    a = [-2 * pi[0], -2 * pi[1], -2 * pi[2], 1, 1, cA * (1 << 22), cB * (1 << 11), cC]
    b = [pj[0], pj[1], pj[2], (nj >> 11) << 11, nj & 2047, 1, 1, 1]
    return a, b


def test_bound_formula_boundaries():
    assert admitted(1023, 9) and not admitted(1024, 9)
    assert admitted(0, 0)
    assert not admitted(1182, 0)


@pytest.mark.parametrize("m", [0, 1, 7, 512, 700, 1000, 1023])
def test_extreme_coordinates_are_exact(m):
    vals = sorted({-m, -m + 1, 0, m - 1, m} & set(range(-m, m + 1)))
    corners = list(itertools.product(vals, repeat=3))
    r2s = [0, 1, 9, 3 * m * m, 3 * m * m + 5, 12 * m * m]
    checked = 0
    for r2e in r2s:
        if r2e > 12 * m * m or not admitted(m, r2e):
            continue
        for pi in corners[:: max(1, len(corners) // 40)]:
            for pj in corners:
                a, b = operands(pi, pj, r2e)
                assert all(sig_bits(v) <= 11 for v in a + b), (pi, pj, r2e, a, b)
                terms = [x * y for x, y in zip(a, b)]
                d2 = sum((u - v) ** 2 for u, v in zip(pi, pj))
                assert sum(terms) == d2 - r2e - 1
                assert sum(abs(t) for t in terms) < (1 << 24), (pi, pj, r2e)
                checked += 1
    assert checked > 0


def test_digit_split_reconstructs_over_the_whole_range():
    for c in list(range(-20000, 20000, 7)) + [-(12 * 1023 ** 2 + 1), 3 * 1023 ** 2, (1 << 24) - 1, -(1 << 24) + 1]:
        cA, cB, cC = balanced_digits(c)
        assert cA * (1 << 22) + cB * (1 << 11) + cC == c
        assert -1024 <= cB <= 1023 and -1024 <= cC <= 1023
        assert abs(cA * (1 << 22)) <= abs(c) + (1 << 21) + 1024
