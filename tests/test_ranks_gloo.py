"""The N > 1 benchmark layout on CPU ranks (gloo, world size 2): each rank
builds its own instance from its own seed, and the only exchange is the MAX
of the timings."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2609_39443_b300 import workloads as W
from paper_2609_39443_b300.ranks import instance_seed, max_over_ranks


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.make_canopy(instance_seed(rank), 2.0, nx=32, ny=32, nz=24, n_sx=2, n_sy=2, n_cv=8, height=0.03)
    t = max_over_ranks([1.0 + rank, 10.0 - rank, float(wl.step.P.sum())], dist)
    out[rank] = (t, float(wl.step.P.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_share_only_the_timing_maximum():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (t0, p0), (t1, p1) = res[0], res[1]
    assert t0[:2] == t1[:2] == [2.0, 10.0]
    assert p0 != p1                                  # independent instances per rank
    assert t0[2] == t1[2] == max(p0, p1)


def test_without_a_group_the_values_pass_through():
    assert max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
