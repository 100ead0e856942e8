"""Replayed gather (AL_OPT_RECORD): the segment pass records the (cell,
segment) pairs of the certified lines and the gather replays them.

The per-pair values are computed by the same explicitly rounded arithmetic
in both passes and every cell sums its sources as fixed-point integers, so a
step gives the same bits whether a brick replays its records, recomputes
them (first step, overflowing region, records off), or runs in a batch.
The replayed steps also match the oracle."""
import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W
from paper_2609_39443_b300.al import (OPT_RECORD, OPT_WEIGHTS, ST_REPLAYED, ST_SUPPORT, WEIGHTS_SEGMENT)

from helpers import BRICK_PASSES, compare

pytestmark = pytest.mark.gpu


def _outs(inst, npts):
    return {"S": inst.S.cpu().numpy().copy(), "F": inst.F[:, :npts].cpu().numpy().copy(),
            "totals": inst.totals.cpu().numpy().copy(), "status": inst.status.cpu().numpy().copy()}


def _run(wl, steps, record, moves=None, bz=None):
    """`steps` steps with the segment weights pass, recording and replaying
    pairs (record True) or gathering them in the same fixed point (False);
    moves[k] (optional) are the positions of step k.  Returns the outputs
    of every step."""
    import torch
    from paper_2609_39443_b300.al import OPT_BRICK_Z, Instance
    inst = Instance(wl, options=BRICK_PASSES)
    inst.grid.set_option(OPT_WEIGHTS, WEIGHTS_SEGMENT)
    inst.grid.set_option(OPT_RECORD, 1 if record else 2)
    if bz:
        inst.grid.set_option(OPT_BRICK_Z, bz)
    out = []
    for k in range(steps):
        if moves is not None:
            inst.set_points(P=moves[k])
        inst.status.zero_()
        inst.step()
        torch.cuda.synchronize()
        out.append(_outs(inst, wl.beams.n_points))
    inst.close()
    return out


def _same(a, b):
    for k in ("S", "F", "totals"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("name", ["canopy", "flume_reduced", "random_fp64"])
def test_replay_equals_gather_bitwise(name):
    if name == "canopy":
        wl = W.make_canopy(4, 2.0)
    elif name == "flume_reduced":
        wl = W.make_flume(2, nx=256, ny=64, nz=128, n_sx=20, n_sy=8)
    else:
        wl = W.make_random(71, 40, 33, 30, n_lines=8, precision="fp64", kinds=("stem", "arc"))
    on, off = _run(wl, 3, True), _run(wl, 3, False)
    for k in range(3):
        _same(on[k], off[k])
        assert on[k]["status"][ST_SUPPORT] == off[k]["status"][ST_SUPPORT]
    # the first step has no regions yet; the later ones replay
    assert on[0]["status"][ST_REPLAYED] == 0 and off[2]["status"][ST_REPLAYED] == 0
    assert on[2]["status"][ST_REPLAYED] > 0
    print(name, "replayed bricks", on[2]["status"][ST_REPLAYED])


def test_replay_matches_the_oracle():
    wl = W.make_canopy(5, 2.0)
    out = _run(wl, 2, True)
    o1 = oracle.point_step(wl.grid, wl.beams, wl.step)
    o2 = oracle.sample_drag_spread(wl, f_prev=o1["f"])
    g = {k: out[1][k].astype(np.float64) if k in ("S", "F") else out[1][k] for k in out[1]}
    m = compare(wl, g, o2, label="replayed canopy")
    assert out[1]["status"][ST_REPLAYED] > 0
    assert out[1]["status"][ST_SUPPORT] == oracle.count_support(wl.grid, wl.beams, wl.step.P)
    print("replayed canopy", m)


def test_moving_beams_and_brick_heights():
    """Beams jump by several cells between steps (their pairs fall in bricks
    whose regions were sized for other counts), at every brick height: the
    bits still equal the recomputed projection's."""
    wl = W.make_random(72, 48, 40, 36, n_lines=10, kinds=("stem", "arc"))
    P0 = wl.step.P.astype(np.float64)
    shift = np.array([3.7, -2.2, 1.3])[:, None] * wl.grid.h
    moves = [P0, P0 + shift, P0 + 2 * shift, P0 + 2 * shift]
    moves = [m.astype(wl.step.P.dtype) for m in moves]
    on, off = _run(wl, 4, True, moves=moves), _run(wl, 4, False, moves=moves)
    for k in range(4):
        _same(on[k], off[k])
    assert on[3]["status"][ST_REPLAYED] > 0
    # the other brick heights (the brick weights pass of the lines without a
    # certificate works relative to the brick corner, so across heights S
    # agrees to rounding, not bit for bit)
    for bz in (4, 16):
        on_z, off_z = _run(wl, 3, True, bz=bz), _run(wl, 3, False, bz=bz)
        for k in range(3):
            _same(on_z[k], off_z[k])
        assert on_z[2]["status"][ST_REPLAYED] > 0


def test_batch_replay_equals_alone():
    import torch
    from paper_2609_39443_b300.al import Batch, Instance
    wls = W.make_batched(6, 4, max_cells=96 * 64 * 64)
    alone, inb = [Instance(w, options=BRICK_PASSES) for w in wls], [Instance(w) for w in wls]
    for x in alone + inb:
        x.grid.set_option(OPT_WEIGHTS, WEIGHTS_SEGMENT)
    for x in alone:
        x.grid.set_option(OPT_RECORD, 2)              # alone recomputes every pair
    batch = Batch(inb, use_graph=True)
    for _ in range(3):
        for a in alone:
            a.status.zero_()
            a.step()
        for b in inb:
            b.status.zero_()
        batch.run()
        torch.cuda.synchronize()
        for a, b in zip(alone, inb):
            for x, y in ((a.S, b.S), (a.F, b.F), (a.totals, b.totals)):
                np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    assert sum(int(b.status[ST_REPLAYED]) for b in inb) > 0
    batch.close()
    for x in alone + inb:
        x.close()


def test_segment_pass_keeps_every_wedge_cell():
    """A random canopy instance with a cell in the wedge behind a node, where
    both segments' feet clamp to the node and its bisector value sits at the
    edge of the FP32 band: the two segments must agree on which keeps it.
    One segment-pass step matches the oracle and its support count."""
    wl = W.make_batched(6, 4, max_cells=96 * 64 * 64)[1]
    out = _run(wl, 2, True)
    o = oracle.sample_drag_spread(wl)
    o1 = oracle.point_step(wl.grid, wl.beams, wl.step)
    o2 = oracle.sample_drag_spread(wl, f_prev=o1["f"])
    for k, ref in ((0, o), (1, o2)):
        g = {key: out[k][key].astype(np.float64) if key in ("S", "F") else out[k][key] for key in out[k]}
        compare(wl, g, ref, label=f"wedge step {k}", sumF_ref="abs")
        assert out[k]["status"][ST_SUPPORT] == oracle.count_support(wl.grid, wl.beams, wl.step.P)
