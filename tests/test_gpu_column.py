"""The column march (AL_OPT_COLUMN): bricks whose lines all climb take both
projection passes by marching up each column of cells.  Checked against the
FP64 oracle element by element (S within 1e-5 of max|S|, the total force and
the resultant within 1e-6), with the number of (cell, line) pairs inside the
3-eps support equal to the oracle's (every closest-segment and cut-off
decision), at every brick height, on bricks that mix column-march lines with
lines that take the brick passes, with zero-weight deposits, over steps that
relax, and bit for bit from run to run."""
import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W

from helpers import compare

pytestmark = pytest.mark.gpu


def _run(wl, column=1, bz=None, steps=1, weights=None):
    import torch
    from paper_2609_39443_b300.al import OPT_BRICK_Z, OPT_COLUMN, OPT_WEIGHTS, Instance
    inst = Instance(wl)
    inst.grid.set_option(OPT_COLUMN, column)
    if bz:
        inst.grid.set_option(OPT_BRICK_Z, bz)
    if weights is not None:
        inst.grid.set_option(OPT_WEIGHTS, weights)
    for _ in range(steps):
        inst.status.zero_()
        inst.step()
    torch.cuda.synchronize()
    out = {"S": inst.S.double().cpu().numpy(), "F": inst.F[:, :wl.beams.n_points].double().cpu().numpy(),
           "totals": inst.totals.cpu().numpy(), "status": inst.status.cpu().numpy()}
    assert out["status"][15] == 0                    # no column-march index guard fired
    nbrick = -(-wl.grid.nx // 16) * -(-wl.grid.ny // 16) * -(-wl.grid.nz // (bz or 8))
    inst.close()
    return out, nbrick


@pytest.mark.parametrize("bz", [4, 8, 16])
@pytest.mark.parametrize("eps_cells", [1.5, 2.0, 3.0])
def test_canopy_column_march_vs_oracle(eps_cells, bz):
    from paper_2609_39443_b300.al import ST_COLUMN, ST_SUPPORT
    wl = W.make_canopy(5, eps_cells, nx=128, ny=96, nz=80, n_sx=8, n_sy=8, n_cv=50, height=0.25)
    g, nbrick = _run(wl, bz=bz)
    o = oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label=f"canopy column eps {eps_cells} bz {bz}")
    assert g["status"][ST_COLUMN] == nbrick          # every brick marched
    assert g["status"][ST_SUPPORT] == oracle.count_support(wl.grid, wl.beams, wl.step.P)
    print("column canopy", eps_cells, bz, m, "refined", g["status"][6])


def test_flume_column_march_vs_oracle():
    from paper_2609_39443_b300.al import ST_COLUMN, ST_SUPPORT
    wl = W.make_flume(3, nx=256, ny=64, nz=128, n_sx=20, n_sy=8)
    g, nbrick = _run(wl, bz=16)
    o = oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label="flume reduced column")
    assert g["status"][ST_COLUMN] == nbrick
    assert g["status"][ST_SUPPORT] == oracle.count_support(wl.grid, wl.beams, wl.step.P)
    print("column flume", m)


@pytest.mark.parametrize("seed", [61, 62, 63])
def test_bricks_mixing_column_and_brick_lines(seed):
    """Stems (column march) next to arcs, random walks and horizontal lines
    (brick passes): bricks with both take the brick passes for every line,
    the others the column march."""
    from paper_2609_39443_b300.al import ST_COLUMN, ST_SUPPORT, WEIGHTS_BRICK, WEIGHTS_SEGMENT
    wl = W.make_random(seed, 64, 48, 40, n_lines=14, kinds=("stem", "stem", "stem", "arc", "random", "flat"),
                       n_cv=(8, 30), has_alpha=seed == 62)
    o = oracle.sample_drag_spread(wl)
    for weights in (WEIGHTS_BRICK, WEIGHTS_SEGMENT):
        g, nbrick = _run(wl, weights=weights)
        compare(wl, g, o, label=f"mixed {seed} w{weights}", sumF_ref="abs")
        assert 0 < g["status"][ST_COLUMN] < nbrick
        assert g["status"][ST_SUPPORT] == oracle.count_support(wl.grid, wl.beams, wl.step.P)
        for k in range(6):
            assert g["status"][k] == o["status"][k]


def test_column_march_on_and_off_agree():
    wl = W.make_canopy(6, 2.0, nx=96, ny=64, nz=72, n_sx=6, n_sy=6, n_cv=40, height=0.2)
    o = oracle.sample_drag_spread(wl)
    on, _ = _run(wl, column=1)
    off, _ = _run(wl, column=0)
    compare(wl, on, o, label="on")
    compare(wl, off, o, label="off")
    assert on["status"][8] == off["status"][8]
    scale = np.abs(o["S"]).max()
    assert np.abs(on["S"] - off["S"]).max() <= 2e-5 * scale


def test_column_march_bitwise_reproducible_over_relaxed_steps():
    wl = W.make_canopy(7, 2.0, nx=96, ny=64, nz=72, n_sx=6, n_sy=6, n_cv=40, height=0.2)
    a, _ = _run(wl, steps=2)
    b, _ = _run(wl, steps=2)
    for k in ("S", "F", "totals"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    o1 = oracle.point_step(wl.grid, wl.beams, wl.step)
    o2 = oracle.sample_drag_spread(wl, f_prev=o1["f"])
    compare(wl, a, o2, label="relaxed column")


def test_column_march_zero_weight_deposits():
    """Quarter-cell segments: nodes with w_k = 0 inside column-march bricks
    deposit their load in their cell."""
    from paper_2609_39443_b300.al import ST_COLUMN
    wl = W.random_canopy(12, 48, 40, 32, 0.005, 60, 64, 1.6, name="fine")
    g, _ = _run(wl)
    o = oracle.sample_drag_spread(wl)
    assert o["status"][4] > 0 and g["status"][4] == o["status"][4]
    assert g["status"][ST_COLUMN] > 0
    compare(wl, g, o, label="fine column")


def test_dense_stems_several_batches_in_a_column_brick():
    """700 stems: more than 32 candidate lines per brick, several batches of
    lines per brick, and more than 512 (several passes over the mask)."""
    from paper_2609_39443_b300.al import ST_COLUMN
    wl = W.random_canopy(11, 64, 48, 32, 0.005, 700, 12, 2.0, name="dense")
    g, _ = _run(wl)
    o = oracle.sample_drag_spread(wl)
    compare(wl, g, o, label="dense column")
    assert g["status"][ST_COLUMN] > 0
    assert g["status"][8] == oracle.count_support(wl.grid, wl.beams, wl.step.P)


def test_tile_stores_and_the_fallback_write_the_same_sources():
    """The spread's S tile leaves by TMA tensor stores when S is 16-byte
    aligned with rows of a multiple of 16 bytes, else by plain stores: an S
    shifted by one float (no descriptor) gets the same bits, and the
    totals agree to rounding."""
    import torch
    from paper_2609_39443_b300.al import Instance
    wl = W.make_flume(2, nx=160, ny=48, nz=64, n_sx=14, n_sy=5, height=0.2)
    a = Instance(wl)
    a.step()
    b = Instance(wl)
    n = wl.grid.n_cells
    raw = torch.empty(3 * n + 1, dtype=torch.float32, device="cuda")
    S = raw[1:].view(3, n)                          # 4 bytes past an aligned start
    b.grid.step(b.U, b.P, b.Pdot, S, b.F, alpha=b.alpha, totals=b.totals, status=b.status)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(S.cpu().numpy(), a.S.cpu().numpy())
    np.testing.assert_array_equal(b.F.cpu().numpy(), a.F.cpu().numpy())
    ta, tb = a.totals.cpu().numpy(), b.totals.cpu().numpy()
    assert np.abs(ta - tb).max() <= 1e-6 * np.abs(ta).max()
    a.close()
    b.close()
