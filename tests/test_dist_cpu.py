"""The multi-process path on CPU (gloo, world size 2): sharding of operating
points across ranks covers every unit exactly once, and the timing reduction
takes the slowest rank. No GPU and no data-path collective are involved."""
import os
import socket

import pytest

from paper_2112_09271_gb300 import dist as pdist


@pytest.mark.parametrize("n,world", [(8, 2), (7, 2), (3, 4), (0, 2), (16, 8)])
def test_shard_partitions_the_units(n, world):
    seen = []
    for r in range(world):
        lo, hi = pdist.shard(n, r, world)
        assert 0 <= lo <= hi <= n
        assert hi - lo in (n // world, n // world + 1)
        seen.extend(range(lo, hi))
    assert seen == list(range(n))


def test_shard_rejects_bad_arguments():
    with pytest.raises(ValueError):
        pdist.shard(4, 2, 2)
    with pytest.raises(ValueError):
        pdist.shard(4, 0, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = pdist.shard(8, rank, world)
        t = 1.0 + rank          # rank 1 is the slow one
        out[rank] = (lo, hi, pdist.max_over_ranks(t), pdist.sum_over_ranks(hi - lo))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_timing_and_units():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()   # no fork of this multi-threaded process
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0][:2] == (0, 4) and out[1][:2] == (4, 8)
    assert out[0][2] == out[1][2] == 2.0      # the slowest rank sets the time
    assert out[0][3] == out[1][3] == 8.0      # every unit counted once
