"""Algorithms 1 and 2 of Section 3 on the GPU (linear-time same-site collisions and
face contacts) against the CPU oracle's Algorithms 1/2 and pairwise counts."""
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


def dev(*a):
    return [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in a]


def run(cc, fn, x, y, z):
    out = fn(*dev(x, y, z))
    torch.cuda.synchronize()
    return cc.as_u64(out)


@pytest.mark.parametrize("n,box", [(0, 4), (1, 4), (2, 1), (500, 4), (2001, 6), (30000, 16), (100000, 40)])
def test_dense_box(cc, n, box):
    rng = np.random.default_rng(n + box)
    x, y, z = (rng.integers(-box, box, n).astype(np.int32) for _ in range(3))
    assert run(cc, cc.count_same_site, x, y, z) == oracle.count_colls(x, y, z)
    assert run(cc, cc.count_contacts, x, y, z) == oracle.count_contacts(x, y, z)


def test_bead_chains(cc):
    """Random chains with unit steps in 6 directions (Section 5's CPU workload)."""
    rng = np.random.default_rng(3)
    steps = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    for n in (64, 1920, 20000):
        ch = np.cumsum(steps[rng.integers(0, 6, n)], axis=0).astype(np.int32)
        x, y, z = ch[:, 0].copy(), ch[:, 1].copy(), ch[:, 2].copy()
        assert run(cc, cc.count_same_site, x, y, z) == oracle.count_colls(x, y, z)
        assert run(cc, cc.count_contacts, x, y, z) == oracle.count_contacts(x, y, z)


def test_hashed_wide_box(cc):
    """A box too large for the dense array: the hash-table path; references are the
    pairwise counts at r2 = 0 and r2 = 1 (contacts = pairs at squared distance 1)."""
    rng = np.random.default_rng(4)
    n = 6000
    base = rng.integers(0, 1_000_000, (n // 3, 3)).astype(np.int32)
    pts = np.concatenate([base, base[: n // 3], base + np.array([1, 0, 0], dtype=np.int32)])
    pts = pts[rng.permutation(len(pts))]
    x, y, z = (pts[:, a].copy() for a in range(3))
    c0 = oracle.count_i32(x, y, z, 0)
    c1 = oracle.count_i32(x, y, z, 1)
    assert run(cc, cc.count_same_site, x, y, z) == c0
    assert run(cc, cc.count_contacts, x, y, z) == c1 - c0


def test_same_cell_full_size(cc):
    s = synth.cfg2(262144, same_cell=True)
    want = oracle.count_colls(s["x"], s["y"], s["z"])
    assert run(cc, cc.count_same_site, s["x"], s["y"], s["z"]) == want
    t = dev(s["x"], s["y"], s["z"])
    pc = cc.count_pairs(*t, r2=0)
    torch.cuda.synchronize()
    assert cc.as_u64(pc) == want


def test_span_too_large(cc):
    x = np.array([0, 3_000_000, 5], dtype=np.int32)
    out = cc.count_same_site(*dev(x, x * 0, x * 0))
    assert cc.stream_status() == cc.CC_ERR_RANGE
    assert cc.as_u64(out) == cc.CC_COUNT_INVALID
