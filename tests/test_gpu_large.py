"""Large sets (beyond what the CPU oracle finishes in seconds).

Closed forms that need no oracle: every site of a 128 x 128 x 64 integer lattice
(2^20 objects, permuted) and of a 128 x 64 x 64 lattice of FP32 spheres (2^19), whose
counts and interaction sums follow from the offsets d with |d|^2 <= r2 and their
multiplicities prod_a (L_a - |d_a|), on the tensor-core forms and on the FP32 pipe.
Random sets: the tensor-core forms against the FP32-pipe kernel, two independent GPU
implementations of the same exact predicate, on 2^20 integer points and 2^19 FP32
spheres (counts equal, sums within 1e-5). At 2^19 points the two halves of a set are
also counted by the batched path (a third kernel) and by the tensor-core kernel.
"""
import itertools
import math

import numpy as np
import pytest

import synth
from tests import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import paper_1901_11204_gb300 as cc
    cc.build()
    cc.lib()
    return cc


def both_kernels(cc, fn):
    out = {}
    for tc in (True, False):
        cc.set_tensor_cores(tc)
        try:
            res = fn()
            torch.cuda.synchronize()
            out[tc] = (res, cc.stream_mode())
        finally:
            cc.set_tensor_cores(True)
    return out


def lattice_count_and_sum(L, r2):
    """Unordered pairs of distinct lattice sites within squared distance r2 and the sum of
    1/|d| over them: half the sums over non-zero offsets d of mult(d) and mult(d)/|d|,
    mult(d) = prod_a max(L_a - |d_a|, 0)."""
    m = math.isqrt(r2)
    cnt, terms = 0, []
    for d in itertools.product(range(-m, m + 1), repeat=3):
        d2 = sum(v * v for v in d)
        if d2 == 0 or d2 > r2:
            continue
        mult = math.prod(max(L[a] - abs(d[a]), 0) for a in range(3))
        cnt += mult
        terms.append(mult / math.sqrt(d2))
    assert cnt % 2 == 0
    return cnt // 2, math.fsum(terms) / 2


def test_lattice_closed_form_2_20(cc):
    """2^20 integer points on every site of a 128 x 128 x 64 box, permuted: counts at
    several radii (sparse hits, walked; dense hits, counted in registers) and the
    interaction sum, on both kernels, against the closed form."""
    L = (128, 128, 64)
    x, y, z = pins.lattice_points(L, np.random.default_rng(20))
    assert len(x) == 1 << 20
    t = [torch.from_numpy(a).cuda() for a in (x, y, z)]
    for r2 in (1, 3, 9):
        want = pins.lattice_pairs_closed_form(L, r2)
        out = both_kernels(cc, lambda: cc.count_pairs(*t, r2=r2))
        (a, ma), (b, mb) = out[True], out[False]
        assert ma == cc.MODE_TENSOR and mb == cc.MODE_FP32_EXACT
        assert cc.as_u64(a) == cc.as_u64(b) == want, (r2, cc.as_u64(a), cc.as_u64(b), want)
    want_c, want_s = lattice_count_and_sum(L, 3)
    out = both_kernels(cc, lambda: cc.interaction_sum(*t, r2=3))
    for tc in (True, False):
        (s, c), _ = out[tc]
        assert cc.as_u64(c) == want_c
        assert abs(float(s.item()) - want_s) <= 1e-5 * want_s, (tc, float(s.item()), want_s)


def test_sphere_lattice_closed_form_2_19(cc):
    """2^19 FP32 spheres centred on every site of a 128 x 64 x 64 box (integer
    coordinates, exact in FP32): radius 0.5 makes face neighbours touch (d^2 = 1 = s^2,
    inclusive), radius 0.75 adds the in-plane diagonals (d^2 = 2 <= 2.25); counts and sums
    against the closed form on both kernels."""
    L = (128, 64, 64)
    xi, yi, zi = pins.lattice_points(L, np.random.default_rng(21))
    x, y, z = (a.astype(np.float32) for a in (xi, yi, zi))
    for rad, r2 in ((0.5, 1), (0.75, 2)):
        r = np.full(len(x), rad, dtype=np.float32)
        t = [torch.from_numpy(a).cuda() for a in (x, y, z, r)]
        want_c, want_s = lattice_count_and_sum(L, r2)
        out = both_kernels(cc, lambda: cc.count_pairs(t[0], t[1], t[2], r=t[3]))
        (a, ma), (b, mb) = out[True], out[False]
        assert ma == cc.MODE_TENSOR_SPHERES and mb == cc.MODE_FP32_SPHERES
        assert cc.as_u64(a) == cc.as_u64(b) == want_c, (rad, cc.as_u64(a), cc.as_u64(b), want_c)
        out = both_kernels(cc, lambda: cc.interaction_sum(t[0], t[1], t[2], r=t[3]))
        for tc in (True, False):
            (s, c), _ = out[tc]
            assert cc.as_u64(c) == want_c
            assert abs(float(s.item()) - want_s) <= 1e-5 * want_s, (rad, tc, float(s.item()), want_s)


def test_integer_points_2_20(cc):
    c = synth.cfg2(1 << 20)
    t = [torch.from_numpy(c[k]).cuda() for k in "xyz"]
    for r2 in (9, 400):
        out = both_kernels(cc, lambda: cc.count_pairs(*t, r2=r2))
        (a, ma), (b, mb) = out[True], out[False]
        assert ma == cc.MODE_TENSOR and mb == cc.MODE_FP32_EXACT
        assert cc.as_u64(a) == cc.as_u64(b) > 0
    out = both_kernels(cc, lambda: cc.interaction_sum(*t, r2=400))
    (sa, ca), ma = out[True]
    (sb, cb), mb = out[False]
    assert cc.as_u64(ca) == cc.as_u64(cb)
    assert abs(float(sa.item()) - float(sb.item())) <= 1e-5 * float(sb.item())


def test_spheres_2_19(cc):
    x, y, z, r = synth.sphere_points(1 << 19, 31)
    t = [torch.from_numpy(a).cuda() for a in (x, y, z, r)]
    out = both_kernels(cc, lambda: cc.count_pairs(t[0], t[1], t[2], r=t[3]))
    (a, ma), (b, mb) = out[True], out[False]
    assert ma == cc.MODE_TENSOR_SPHERES and mb == cc.MODE_FP32_SPHERES
    assert cc.as_u64(a) == cc.as_u64(b) > 0
    out = both_kernels(cc, lambda: cc.interaction_sum(t[0], t[1], t[2], r=t[3]))
    (sa, ca), _ = out[True]
    (sb, cb), _ = out[False]
    assert cc.as_u64(ca) == cc.as_u64(cb)
    assert abs(float(sa.item()) - float(sb.item())) <= 1e-5 * float(sb.item())


def test_split_property_2_19(cc):
    """The halves of a 2^19-point set counted by the tensor-core kernel equal the same
    halves counted by the batched path; the whole set's count agrees between the two
    single-set kernels and exceeds the halves' sum (the cross pairs)."""
    c = synth.cfg2(1 << 19)
    h = 1 << 18
    t = [torch.from_numpy(c[k]).cuda() for k in "xyz"]
    whole = cc.as_u64(cc.count_pairs(*t, r2=25))
    lo = cc.as_u64(cc.count_pairs(*(a[:h] for a in t), r2=25))
    hi = cc.as_u64(cc.count_pairs(*(a[h:] for a in t), r2=25))
    torch.cuda.synchronize()
    assert cc.stream_mode() == cc.MODE_TENSOR
    off = torch.tensor([0, h, 1 << 19], dtype=torch.int64, device="cuda")
    plan = cc.Plan(2, 1 << 19)
    counts, _ = plan.count_pairs_batched(*t, off, r2=25)
    torch.cuda.synchronize()
    plan.close()
    assert [int(v) for v in counts.cpu().numpy().view(np.uint64)] == [lo, hi]
    cc.set_tensor_cores(False)
    try:
        whole_fp32 = cc.as_u64(cc.count_pairs(*t, r2=25))
        torch.cuda.synchronize()
    finally:
        cc.set_tensor_cores(True)
    assert whole == whole_fp32 and whole > lo + hi
