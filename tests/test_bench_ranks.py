"""Host logic of the multi-replica bench path on two gloo ranks (CPU): the whole-job
time is the slowest rank's and the work is summed over ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [1.5, 2.5][rank]
    work = [1.0e6, 3.0e6][rank]
    t, w = bench.aggregate_over_ranks(dist, elapsed, work, "cpu")
    out[rank] = (t, w)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        assert out[r] == (2.5, 4.0e6)
    assert bench_value(out[0]) == pytest.approx(1.6e6)


def bench_value(res):
    t, w = res
    return w / t


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(None, 3.0, 7.0, "cpu") == (3.0, 7.0)
