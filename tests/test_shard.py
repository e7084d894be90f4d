"""Host-side logic of the N>1 path, on CPU: the cell partition and the
fixed-order theta-gradient reduction across two gloo ranks."""
import os
import socket

import numpy as np
import pytest

from paper_2501_00011_gb300 import shard


@pytest.mark.parametrize("n,world", [(0, 1), (1, 2), (10_000, 1), (10_000, 8), (50_001, 4), (7, 3), (3, 8)])
def test_cell_range_partitions(n, world):
    ranges = [shard.cell_range(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


def test_cell_range_rejects_bad_requests():
    for args in [(10, 2, 2), (10, -1, 2), (10, 0, 0), (-1, 0, 1)]:
        with pytest.raises(ValueError):
            shard.cell_range(*args)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(100 + rank)
        g = rng.standard_normal(186) * 10.0 ** rng.integers(-12, 3, 186)
        tot = shard.reduce_theta_grad(g)
        import torch
        tot_t = shard.reduce_theta_grad(torch.from_numpy(g))
        q.put((rank, g, tot, tot_t.numpy()))
    finally:
        dist.destroy_process_group()


def test_theta_reduction_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g0, g1 = out[0][1], out[1][1]
    expect = g0 + g1                      # rank order 0 then 1
    for rank, g, tot, tot_t in out:
        assert np.array_equal(tot, expect) and np.array_equal(tot_t, expect)
