"""The multi-GPU mode of the benchmark is replicas only: each rank solves its
own system and the job's throughput is all ranks' bytes over the slowest
rank's time.  Exercised here with world size 2 on the gloo backend (CPU),
which needs no GPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_bytes = [3.0e9, 5.0e9][rank]
        local_ms = [200.0, 250.0][rank]
        value, ms, total = bench.replica_throughput(local_bytes, local_ms, dist, "cpu")
        q.put((rank, value, ms, total))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_world2_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, value, ms, total in res:
        assert ms == 250.0 and total == 8.0e9
        assert value == pytest.approx(8.0e9 / 0.25 / 1e9)


def test_replica_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    value, ms, total = bench.replica_throughput(4.0e9, 100.0)
    assert (value, ms, total) == (40.0, 100.0, 4.0e9)
