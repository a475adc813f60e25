"""bench.py's multi-rank aggregation on CPU (gloo, two ranks, no GPU)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r timed (r + 1) seconds and ran 10 (r + 1) iterations
    el, it = bench.aggregate(float(rank + 1), 10 * (rank + 1), world, "cpu")
    out[rank] = (el, it)
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    # max time over ranks, sum of iterations: value = 30 iterations / 2 s
    assert res[0] == res[1] == (2.0, 30.0)


def test_aggregate_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(1.5, 7, 1, "cpu") == (1.5, 7.0)
