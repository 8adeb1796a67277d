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


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the oracle arm) prints one JSON line with
    the contract's keys, on the host cores, without a GPU (here on the 40^3
    cavity; the arm times the first steps of the workload it is given)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--workload", "cavity3d_40"], capture_output=True, text=True, cwd=root,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["config"]["same_config"] is True and d["config"]["cells"] == 40 ** 3
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
