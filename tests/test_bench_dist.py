"""Host logic of the multi-process benchmark path on CPU (gloo, world size 2):
max-over-ranks timing and the whole-job throughput; the reference arm runs on
rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [200.0, 250.0][rank]
    ms, value = bench.aggregate(1_000_000, ms_local, world, dist)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate_takes_slowest_rank():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        ms, value = out[r]
        assert ms == 250.0
        assert value == pytest.approx(2 * 1_000_000 / 0.25)


def test_single_process_aggregate():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ms, v = bench.aggregate(4096, 5.0, 1, None)
    assert ms == 5.0 and v == pytest.approx(4096 / 0.005)
