"""The bench's multi-rank arithmetic (replicas: summed work, slowest-rank time) on two gloo
ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        entries = 1000.0 * (rank + 1)        # rank 0: 1000 entries, rank 1: 2000
        ms = 10.0 * (rank + 1)               # rank 0: 10 ms, rank 1: 20 ms
        v = bench.job_throughput(ws, entries, ms, device="cpu")
        mx = bench.max_over_ranks(ws, ms, device="cpu")
        out[rank] = (v, mx)
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_throughput():
    import torch.multiprocessing as mp
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    # 3000 entries over the slowest rank's 20 ms
    for rank in range(ws):
        v, mx = res[rank]
        assert mx == 20.0
        assert abs(v - 3000.0 / 0.020) < 1e-6
