"""The bench's multi-rank aggregation (replicas per rank, max time over ranks) on world_size 2 with
gloo on the CPU."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    ms = bench.max_over_ranks(10.0 + rank, device="cpu")
    out[rank] = (ms, bench.job_value(2, 1000, ms))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 11.0               # slowest rank's time
    assert abs(res[0][1] - 2 * 1000 / 0.011) < 1e-6     # total solves of both replicas / that time
