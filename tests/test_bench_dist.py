"""The multi-process path of bench.py on CPU: two gloo ranks (world size 2)
use the same helpers the GPU ranks use under torchrun - barrier, the slowest
rank's time and the exact sum of the ranks' partial counts (each rank counts
its share of the start vertices) - so `value` = all matches / the slowest
rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo")
    try:
        bench.barrier(world)
        ms = [12.5, 20.0][rank]           # this rank's step time
        matches = [1000, 3000][rank]      # this rank's matches
        slowest = bench.max_over_ranks(world, ms)
        total = bench.sum_over_ranks(world, matches)
        # partial 128-bit counts whose sums carry across 32- and 64-bit limbs
        parts = [[2**64 - 1, 2**32 - 1, 5, 0], [1, 1, 2**100 + 7, 2**127]][rank]
        counts = bench.sum_counts_over_ranks(world, parts)
        out[rank] = (slowest, total, total / (slowest / 1e3), counts)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_torchrun():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, total, value, counts = res[0]
    assert slowest == 20.0 and total == 4000
    assert value == pytest.approx(4000 / 0.020)
    assert counts == [2**64, 2**32, 2**100 + 12, 2**127]


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(1, 3.5) == 3.5
    assert bench.sum_over_ranks(1, 7) == 7
    assert bench.sum_counts_over_ranks(1, [3, 2**70]) == [3, 2**70]
    bench.barrier(1)
