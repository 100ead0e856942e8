"""One grid split along x over two CPU ranks (gloo, world size 2), with the
library's own host-side decomposition (al_slab_plan, local workloads) and
the FP64 oracle computing each rank's share: each rank samples and drags
its lines on its local grid, sums its owned cells' part of the nodal
weights, the ranks add those partial sums (all-reduce), and each rank
spreads into its owned cells with the summed weights (Sec. 3.2.5).  The
assembled S and the owned points' forces equal the monolithic oracle's."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2609_39443_b300 import slab
from paper_2609_39443_b300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _workload(kind):
    if kind == "canopy":
        return W.make_canopy(5, 2.0, nx=128, ny=48, nz=40, n_sx=6, n_sy=3, n_cv=24, height=0.12)
    # lines of every shape, some crossing the slab boundary, one on it
    return W.make_random(17, 96, 40, 36, n_lines=12, kinds=("stem", "arc", "random", "flat"), n_cv=(6, 30))


def _worker(rank, world, port, kind, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = _workload(kind)
    p = slab.plan(wl, world, rank)
    lw = slab.local_workload(wl, p)
    ps = oracle.point_step(lw.grid, lw.beams, lw.step)
    Ps = lw.step.P if lw.step.P_spread is None else lw.step.P_spread
    a, b = p.x0 - p.lx0, p.x1 - p.lx0
    # the slab's partial weights, added over the global point index
    w = torch.zeros(wl.beams.n_points, dtype=torch.float64)
    w[torch.as_tensor(p.points)] = torch.as_tensor(oracle.project_slab(lw.grid, lw.beams, Ps, ps["F"], a, b)["w"])
    dist.all_reduce(w)
    S = oracle.project_slab(lw.grid, lw.beams, Ps, ps["F"], a, b, w.numpy()[p.points])["S"]
    S = S.reshape(3, lw.grid.nz, lw.grid.ny, lw.grid.nx)[..., a:b]
    own = p.owner[p.points] == rank
    out[rank] = (p.x0, p.x1, S, p.points[own], ps["F"][:, own], len(p.lines), p.halo)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["canopy", "mixed"])
def test_two_slabs_equal_the_monolithic_oracle(kind):
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, kind, out), nprocs=world, join=True)
        res = dict(out)
    wl = _workload(kind)
    mono = oracle.sample_drag_spread(wl)
    g = wl.grid
    S = np.zeros((3, g.nz, g.ny, g.nx))
    F = np.full((3, wl.beams.n_points), np.nan)
    for r in range(world):
        x0, x1, Sr, idx, Fr, nl, halo = res[r]
        assert halo % 16 == 0 and nl > 0
        S[..., x0:x1] = Sr
        F[:, idx] = Fr
    assert res[0][1] == res[1][0] and res[0][0] == 0 and res[1][1] == g.nx     # the slabs tile the grid
    Sm = mono["S"].reshape(S.shape)
    scale = np.abs(Sm).max()
    assert scale > 0
    assert np.abs(S - Sm).max() <= 1e-12 * scale
    assert not np.isnan(F).any()                          # every point has an owner
    assert np.abs(F - mono["F"]).max() <= 1e-12 * np.abs(mono["F"]).max()
    # and both slabs carry a share of the sources
    assert np.abs(S[..., :res[0][1]]).max() > 0 and np.abs(S[..., res[0][1]:]).max() > 0


def test_plan_is_checked():
    from paper_2609_39443_b300.al import ALError
    wl = _workload("canopy")
    with pytest.raises(ALError):
        slab.plan(wl, 2, 2)
    p = [slab.plan(wl, 3, r) for r in range(3)]
    assert [q.x0 for q in p] == [0, p[0].x1, p[1].x1] and p[2].x1 == wl.grid.nx
    assert all(q.x0 % 16 == 0 for q in p)
    assert all(q.lx0 <= q.x0 and q.lx1 >= q.x1 for q in p)
    own = p[0].owner
    assert set(np.unique(own)) <= {0, 1, 2}
