"""Batched sets (one graph-captured persistent launch) against the CPU oracle and
against one plain single-set launch per set."""
import json

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import paper_1901_11204_gb300 as cc
    cc.build()
    cc.lib()
    return cc


def to_dev(*a):
    return [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in a]


def make_sets(sizes, seed, box=16, f32=False):
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    n = int(off[-1])
    if f32:
        x, y, z = (rng.random(n).astype(np.float32) * np.float32(0.2) for _ in range(3))
        r = (0.005 + 0.01 * rng.random(n)).astype(np.float32)
        return x, y, z, r, off
    x, y, z = (rng.integers(0, box, n).astype(np.int32) for _ in range(3))
    return x, y, z, None, off


SIZES = [0, 1, 2, 3, 4, 5, 16, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 511, 512, 513,
         1000, 2047, 2048, 2049, 8191, 8192, 8193, 0, 1, 70000]


def test_int_sets_parity(cc):
    x, y, z, _, off = make_sets(SIZES, 1, box=24)
    plan = cc.Plan(len(SIZES), len(x))
    t = to_dev(x, y, z, off)
    for r2 in (0, 4, 25):
        counts, _ = plan.count_pairs_batched(*t[:3], t[3], r2=r2)
        torch.cuda.synchronize()
        want = oracle.count_i32_sets(x, y, z, off, r2)
        assert np.array_equal(counts.cpu().numpy().view(np.uint64), want), r2
    plan.close()


def test_f32_sets_parity_with_sums(cc):
    x, y, z, r, off = make_sets(SIZES[:-1], 2, f32=True)
    plan = cc.Plan(len(SIZES), len(x))
    t = to_dev(x, y, z, r, off)
    counts, sums = plan.count_pairs_batched(*t[:3], t[4], r=t[3], want_sum=True)
    torch.cuda.synchronize()
    wc, ws = oracle.count_f32_sets(x, y, z, r, off)
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), wc)
    got = sums.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, ws, rtol=1e-5, atol=0)
    plan.close()


def test_batched_equals_plain_launches(cc):
    x, y, z, _, off = make_sets([5, 40, 300, 2, 1025, 7, 4096], 3, box=20)
    plan = cc.Plan(16, len(x))
    t = to_dev(x, y, z, off)
    counts, _ = plan.count_pairs_batched(*t[:3], t[3], r2=9)
    torch.cuda.synchronize()
    for k in range(len(off) - 1):
        a, b = int(off[k]), int(off[k + 1])
        single = cc.count_pairs(t[0][a:b], t[1][a:b], t[2][a:b], r2=9)
        assert cc.as_u64(single) == int(counts[k].item()) & 0xFFFFFFFFFFFFFFFF
    plan.close()


def test_replay_with_new_inputs(cc):
    plan = cc.Plan(64, 200000)
    for seed in range(3):
        sizes = np.random.default_rng(seed).integers(0, 3000, 40)
        x, y, z, _, off = make_sets(sizes, 10 + seed, box=30)
        t = to_dev(x, y, z, off)
        counts, _ = plan.count_pairs_batched(*t[:3], t[3], r2=16)
        torch.cuda.synchronize()
        assert np.array_equal(counts.cpu().numpy().view(np.uint64), oracle.count_i32_sets(x, y, z, off, 16))
    plan.close()


def test_range_error_marks_only_that_set(cc):
    x, y, z, _, off = make_sets([10, 20, 30], 4, box=10)
    x = x.copy()
    x[off[1] + 3] = 50000   # set 1 spans more than 32767 on x
    plan = cc.Plan(4, len(x))
    t = to_dev(x, y, z, off)
    counts, _ = plan.count_pairs_batched(*t[:3], t[3], r2=4)
    torch.cuda.synchronize()
    got = counts.cpu().numpy().view(np.uint64)
    want = oracle.count_i32_sets(x, y, z, off, 4)
    assert got[1] == np.uint64(cc.CC_COUNT_INVALID)
    assert got[0] == want[0] and got[2] == want[2]
    plan.close()


def test_custom_band_table_same_results(cc):
    x, y, z, _, off = make_sets(SIZES, 5, box=24)
    t = to_dev(x, y, z, off)
    want = oracle.count_i32_sets(x, y, z, off, 9)
    tables = [
        None,
        {"bands": [{"n_max": 16, "r": 1, "sc": 1}, {"n_max": 1000, "r": 4, "sc": 2},
                   {"n_max": -1, "r": 2, "sc": 0}]},
        {"bands": [{"n_max": -1, "r": 4, "sc": 3}]},
        {"bands": [{"n_max": -1, "r": 1, "sc": 0}]},
        {"bands": [{"n_max": 32, "r": 0, "sc": 0}, {"n_max": -1, "r": 2, "sc": 5}]},
        {"bands": [{"n_max": 256, "r": 0, "sc": 0}, {"n_max": -1, "r": 4, "sc": 2}]},
        {"bands": [{"n_max": 64, "r": 0, "sc": 0}, {"n_max": 128, "r": 1, "sc": 1},
                   {"n_max": 200, "r": 0, "sc": 0}, {"n_max": -1, "r": 2, "sc": 0}]},
    ]
    for tb in tables:
        plan = cc.Plan(len(SIZES), len(x), json.dumps(tb) if tb else None)
        counts, _ = plan.count_pairs_batched(*t[:3], t[3], r2=9)
        torch.cuda.synchronize()
        assert np.array_equal(counts.cpu().numpy().view(np.uint64), want), tb
        plan.close()


def test_cfg4_full(cc):
    c = synth.cfg4()
    off = c["offsets"]
    plan = cc.Plan(len(off) - 1, len(c["x"]))
    t = to_dev(c["x"], c["y"], c["z"], off)
    counts, _ = plan.count_pairs_batched(*t[:3], t[3], r2=25)
    torch.cuda.synchronize()
    want = oracle.count_i32_sets(c["x"], c["y"], c["z"], off, 25)
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), want)
    assert plan.last_items() > 0
    plan.close()


def test_plan_memory_is_bounded(cc):
    """A plan for 4096 sets of up to 2^24 points in all reserves its work queue for at most
    max(tiles, 16384) items per set: a few hundred MB, not a queue that grows with n^2."""
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    plan = cc.Plan(4096, 1 << 24, cc.default_tune_table())
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    plan.close()
    assert used < (512 << 20), used


WARP_SET_TABLE = {"bands": [{"n_max": 32, "r": 0, "sc": 0}, {"n_max": 256, "r": 0, "sc": 0},
                            {"n_max": -1, "r": 2, "sc": 4}]}


def test_warp_per_set_path_all_modes(cc):
    """Sets of 33..256 objects on the one-warp-per-set path (band r = 0 up to 256): integer
    sets in a narrow box (fast exact form) and a wide one (int difference form), counts and
    interaction sums at several radii, and FP32 spheres with sums, against the oracle; sizes
    around the warp multiples, odd and even, and on both sides of the path's limit."""
    sizes = [33, 34, 47, 63, 64, 65, 95, 96, 97, 128, 129, 200, 255, 256, 257, 300, 2, 31, 32]
    tb = json.dumps(WARP_SET_TABLE)
    for box, radii in ((24, (0, 9, 400)), (5000, (250000, 4000000))):
        x, y, z, _, off = make_sets(sizes, 11 + box, box=box)
        t = to_dev(x, y, z, off)
        plan = cc.Plan(len(sizes), len(x), tb)
        for r2 in radii:
            counts, sums = plan.count_pairs_batched(*t[:3], t[3], r2=r2, want_sum=True)
            torch.cuda.synchronize()
            want = oracle.count_i32_sets(x, y, z, off, r2)
            assert np.array_equal(counts.cpu().numpy().view(np.uint64), want), (box, r2)
            ws = np.array([oracle.sum_i32(x[a:b], y[a:b], z[a:b], r2)[1] for a, b in zip(off[:-1], off[1:])])
            np.testing.assert_allclose(sums.cpu().numpy().astype(np.float64), ws, rtol=1e-5, atol=0)
        plan.close()
    x, y, z, r, off = make_sets(sizes, 17, f32=True)
    t = to_dev(x, y, z, r, off)
    plan = cc.Plan(len(sizes), len(x), tb)
    counts, sums = plan.count_pairs_batched(*t[:3], t[4], r=t[3], want_sum=True)
    torch.cuda.synchronize()
    wc, ws = oracle.count_f32_sets(x, y, z, r, off)
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), wc)
    np.testing.assert_allclose(sums.cpu().numpy().astype(np.float64), ws, rtol=1e-5, atol=0)
    plan.close()


def test_band_table_rejects_bad_warp_set_bands(cc):
    """A one-warp-per-set band (r = 0) above the path's 256 objects, or as the last band
    (which takes every larger set), is refused when the plan is created."""
    bad = [{"bands": [{"n_max": 257, "r": 0, "sc": 0}, {"n_max": -1, "r": 2, "sc": 4}]},
           {"bands": [{"n_max": 32, "r": 0, "sc": 0}]},
           {"bands": [{"n_max": 64, "r": 1, "sc": 1}, {"n_max": -1, "r": 0, "sc": 0}]}]
    for tb in bad:
        with pytest.raises(Exception):
            cc.Plan(4, 100, json.dumps(tb))
