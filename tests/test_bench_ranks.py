"""The multi-GPU mode of bench.py runs independent replicas (one lattice per
rank, no exchange between lattices).  Its only collective is the max-reduction
of the timed region; this checks it with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank          # rank 1 is the slowest
    value, ms = bench.aggregate_over_ranks(1000, 10, ms_local, world, dist)
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, ms = res[rank]
        assert ms == pytest.approx(150.0)
        # whole-job rate: all ranks' site updates over the slowest rank's time
        assert value == pytest.approx(2 * 1000 * 10 / 0.150 / 1e9)


def test_single_rank_needs_no_collective():
    import bench
    value, ms = bench.aggregate_over_ranks(1000, 10, 100.0, 1, None)
    assert ms == 100.0 and value == pytest.approx(1000 * 10 / 0.1 / 1e9)
