"""The split along x through the CUDA path (al_step_begin / al_weights_get /
al_weights_set / al_step_end with AL_OPT_OWN_X0/X1), the ranks run one
after the other on one GPU in this process (no kernel of one waits for
another's): the partial weights of the slabs add up over the global point
index, and the assembled S and the owned points' forces match the FP64
oracle at the FP32 tolerances, over two relaxed steps."""
import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import slab
from paper_2609_39443_b300 import workloads as W

from helpers import TOL_S_FP32, TOL_SUMF_FP32

pytestmark = pytest.mark.gpu


def _run(wl, world, steps=1):
    import torch
    ranks = [slab.SlabRank(wl, world, r) for r in range(world)]
    for _ in range(steps):
        for r in ranks:
            r.begin()
        glob = torch.zeros(wl.beams.n_points, dtype=torch.int64, device="cuda")
        for r in ranks:
            r.partial(glob)
        for r in ranks:
            r.end(glob)
    torch.cuda.synchronize()
    g = wl.grid
    S = np.zeros((3, g.nz, g.ny, g.nx))
    F = np.full((3, wl.beams.n_points), np.nan)
    status = np.zeros(16, dtype=np.int64)
    for r in ranks:
        S[..., r.plan.x0:r.plan.x1] = r.owned_S()
        idx, Fr = r.owned_F()
        F[:, idx] = Fr
        status += r.inst.status.cpu().numpy()
        r.close()
    return S, F, status, [r.plan for r in ranks]


def _check(wl, S, F, o):
    Sm = o["S"].reshape(S.shape)
    scale = np.abs(Sm).max()
    assert np.abs(S - Sm).max() <= TOL_S_FP32 * scale, np.abs(S - Sm).max() / scale
    assert not np.isnan(F).any()
    assert np.abs(F - o["F"]).max() <= TOL_SUMF_FP32 * np.abs(o["F"]).max() * 10
    # the resultant: every cell of S written once over the slabs
    V = wl.grid.h ** 3
    tot = S.reshape(3, -1).sum(axis=1) * V
    assert np.abs(tot + o["F"].sum(axis=1)).max() <= 1e-5 * np.abs(o["F"]).sum()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_match_the_oracle(world):
    from paper_2609_39443_b300.al import ST_COLUMN
    wl = W.make_canopy(5, 2.0, nx=160, ny=48, nz=48, n_sx=8, n_sy=3, n_cv=30, height=0.15)
    S, F, status, plans = _run(wl, world)
    _check(wl, S, F, oracle.sample_drag_spread(wl))
    assert status[ST_COLUMN] > 0                       # owned bricks took the column march
    assert all(p.x1 > p.x0 for p in plans)


def test_slabs_with_lines_of_every_shape_over_two_steps():
    """Arcs, random walks and flat lines beside stems (the brick passes for
    their bricks) and relaxation against each rank's previous forces."""
    wl = W.make_random(17, 96, 40, 36, n_lines=12, kinds=("stem", "arc", "random", "flat"), n_cv=(6, 30))
    S, F, _, _ = _run(wl, 2, steps=2)
    o1 = oracle.point_step(wl.grid, wl.beams, wl.step)
    o2 = oracle.sample_drag_spread(wl, f_prev=o1["f"])
    _check(wl, S, F, o2)


def test_a_slab_refuses_what_it_cannot_take():
    from paper_2609_39443_b300.al import OPT_OWN_X0, OPT_OWN_X1, ALError, Batch, Instance
    wl = W.make_canopy(6, 2.0, nx=64, ny=32, nz=32, n_sx=2, n_sy=2, n_cv=10, height=0.1)
    inst = Instance(wl)
    with pytest.raises(ALError):
        inst.grid.set_option(OPT_OWN_X0, 8)            # not a brick column
    with pytest.raises(ALError):
        inst.grid.set_option(OPT_OWN_X1, 40)
    inst.grid.set_option(OPT_OWN_X0, 16)
    with pytest.raises(ALError):
        Batch([inst])                                  # batches take whole grids
    inst.close()
    refl = Instance(W.with_reflect(wl, W.REFLECT_Z_LO), options={OPT_OWN_X1: 32})
    with pytest.raises(ALError):
        refl.step()                                    # no reflecting face on a slab
    refl.close()
