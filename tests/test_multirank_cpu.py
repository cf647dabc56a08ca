"""The N > 1 bench path on CPU ranks (gloo, world size 2): every rank runs its
own independent solves (replicas, no data-path collective); the timed region
is reduced with a max over ranks and the rate counts all ranks' updates."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    el = 1.0 + rank                       # rank 1 is the slower one
    m = bench.reduce_max(el, dist)
    rate = bench.whole_job_rate(1000, world, 10, m)
    out[rank] = (m, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (2.0, 1000 * 2 * 10 / 2.0)
