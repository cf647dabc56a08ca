"""The slab decomposition's host-side exchange on CPU ranks (gloo, world
size 2 and 3): particles are routed to the rank that owns their row after a
move, nothing is lost or duplicated, and the halo rows a rank receives are
its neighbours' boundary rows of the global array."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1808_03801_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _state(w, n, seed):
    pos, vel, pid = W.bimaxwellian(n, seed=seed, y_range=(w["grid"]["lo"][1], w["grid"]["hi"][1]),
                                   x_range=(w["grid"]["lo"][0], w["grid"]["hi"][0]))
    return {"pos": pos, "vel": vel, "pid": pid}


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1808_03801_gb300 import decomp as D
    w = W.cavity(n=12, ppc=10, precision="fp32")
    G = _state(w, 5000, seed=3)
    mine = D.split(G, w, world)[rank]
    # a move: every particle shifted along y by up to two rows, kept in the box
    dy = (w["grid"]["hi"][1] - w["grid"]["lo"][1]) / w["grid"]["ny"]
    rng = np.random.default_rng(100 + rank)
    mine["pos"] = mine["pos"].copy()
    mine["pos"][:, 1] = np.clip(mine["pos"][:, 1] + rng.uniform(-2, 2, len(mine["pid"])) * dy,
                                w["grid"]["lo"][1], np.nextafter(w["grid"]["hi"][1], 0))
    moved = [None] * world
    dist.all_gather_object(moved, mine)
    after = D.exchange_particles(mine, w, world, rank, dist)
    rows = np.arange(w["grid"]["ny"] // world)[:, None] + rank * (w["grid"]["ny"] // world) + np.zeros((1, 4))
    lo, hi = D.exchange_halo(rows, rank, world, dist)
    out[rank] = (after, moved, lo, hi)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_routes_every_particle_once(world):
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    from paper_1808_03801_gb300 import decomp as D
    w = W.cavity(n=12, ppc=10, precision="fp32")
    moved = out[0][1]
    allpos = np.concatenate([m["pos"] for m in moved])
    allpid = np.concatenate([m["pid"] for m in moved])
    owner = D.owner_rows(allpos, w, world)
    got = []
    for r in range(world):
        after = out[r][0]
        assert np.all(D.owner_rows(after["pos"], w, world) == r)
        assert set(after["pid"].tolist()) == set(allpid[owner == r].tolist())
        got.append(after["pid"])
    got = np.concatenate(got)
    assert len(got) == len(allpid) and len(np.unique(got)) == len(got)
    rows_per = w["grid"]["ny"] // world
    for r in range(world):
        lo, hi = out[r][2], out[r][3]
        if r == 0:
            assert lo is None
        else:
            assert np.all(lo == r * rows_per - 1)
        if r == world - 1:
            assert hi is None
        else:
            assert np.all(hi == (r + 1) * rows_per)
