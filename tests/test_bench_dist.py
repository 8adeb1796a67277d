"""Host logic of the multi-rank benchmark path on CPU: two gloo ranks take
the maximum of their timings and meet at the barriers (replicas only; the
solver itself has no collective)."""
import os
import socket

import pytest
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench

    class A:
        impl = "reference"
    ws, r, local = bench.dist_setup(A())
    bench.barrier(ws)
    v = bench.allmax(ws, float(10 + 5 * rank), "cpu")
    bench.barrier(ws)
    out[rank] = (ws, r, v)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_barrier():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == (2, 0, 15.0) and res[1] == (2, 1, 15.0)
