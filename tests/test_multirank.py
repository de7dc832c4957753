"""The N>1 path of bench.py on CPU: world_size 2 over gloo (no GPU).

Every rank counts its own independently drawn sets (no data-path collective); the only
exchange is the max over ranks of the timings, and the whole-job value is the pair
tests of all ranks over the slowest rank's time.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    mine = [10.0 + rank, 3.0 * (rank + 1)]
    got = bench.max_over_ranks(mine, dist, "cpu")
    sets = bench.step_inputs(rank)
    sizes = [len(s[0]) for s in sets]
    # a tiny slice of this rank's first set, counted by the oracle, is exchanged only to
    # check that ranks really hold different inputs
    x, y, z, r2 = sets[0]
    c = oracle.count_i32(x[:3000], y[:3000], z[:3000], 400)
    allc = [None] * world
    dist.all_gather_object(allc, (int(x[:64].sum()), c))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, sizes, allc))


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, got, sizes, allc in out:
        assert got == [11.0, 6.0]
        assert sizes == [262144, 262145, 262144]
        assert allc[0][0] != allc[1][0]   # independent inputs per rank
    import bench
    v = bench.aggregate_value(100, 2, 5, 11.0)
    assert v == pytest.approx(100 * 2 * 5 / 11e-3 / 1e9)
