"""Large sets (beyond what the CPU oracle finishes in seconds): the tensor-core forms
against the FP32-pipe kernel, two independent GPU implementations of the same exact
predicate, on 2^20 integer points and 2^19 FP32 spheres. Counts must be equal; sums
within 1e-5. At 2^19 points the two halves of a set are also counted by the batched
path (a third kernel) and by the tensor-core kernel, which must agree.
"""
import numpy as np
import pytest

import synth

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
