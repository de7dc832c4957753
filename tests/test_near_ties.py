"""FP32 near-tie sphere pairs (tests/golden/f32_near_ties.txt).

CPU: the oracle follows the specified rounding on every pair (exact rationals rounded
step by step), and the fixture really separates that rounding from fused multiply-adds
and from exact arithmetic. GPU: every path (single set, batched, serving) gives the
oracle's count on these pairs, which fails if any kernel contracts the predicate.
"""
import numpy as np
import pytest

import oracle
from tests import pins
from tests.golden import make_near_ties as nt


def test_fixture_separates_roundings():
    pts = nt.load()
    diff = 0
    for k in range(0, len(pts), 2):
        a, b = [float(v) for v in pts[k]], [float(v) for v in pts[k + 1]]
        spec, others = nt.decisions(a, b)
        assert oracle.collide_f32(a, b) == spec == pins._spec_pred_exact(a, b)
        assert oracle.collide_f32(b, a) == spec
        diff += any(o != spec for o in others)
    assert diff == len(pts) // 2


def test_oracle_count_is_per_pair_sum():
    pts = nt.load()
    x, y, z, r = (np.ascontiguousarray(pts[:, i]) for i in range(4))
    want = sum(oracle.collide_f32(pts[k], pts[k + 1]) for k in range(0, len(pts), 2))
    assert oracle.count_f32(x, y, z, r)[0] == want


@pytest.mark.gpu
def test_gpu_paths_follow_specified_rounding():
    torch = pytest.importorskip("torch")
    import paper_1901_11204_gb300 as cc
    cc.build()
    pts = nt.load()
    x, y, z, r = (np.ascontiguousarray(pts[:, i]) for i in range(4))
    want_c, want_s = oracle.count_f32(x, y, z, r)
    t = [torch.from_numpy(a).cuda() for a in (x, y, z, r)]
    got = cc.count_pairs(t[0], t[1], t[2], r=t[3])
    s, c = cc.interaction_sum(t[0], t[1], t[2], r=t[3])
    torch.cuda.synchronize()
    assert cc.as_u64(got) == want_c and cc.as_u64(c) == want_c
    assert abs(float(s.item()) - want_s) <= 1e-5 * abs(want_s)
    # one set per pair through the batched path
    off = np.arange(0, len(x) + 1, 2, dtype=np.int64)
    plan = cc.Plan(len(off) - 1, len(x))
    counts, _ = plan.count_pairs_batched(t[0], t[1], t[2], torch.from_numpy(off).cuda(), r=t[3])
    torch.cuda.synchronize()
    want = np.array([oracle.collide_f32(pts[k], pts[k + 1]) for k in range(0, len(pts), 2)], dtype=np.uint64)
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), want)
    plan.close()
    # through the server
    srv = cc.Server(1 << 28, 64)
    sid = srv.register_set(x, y, z, r=r)
    srv.submit(sid, cc.CC_OP_COUNT, 0, 1)
    srv.drain(30)
    res = srv.poll()
    assert res[0]["count"] == want_c
    srv.close()
