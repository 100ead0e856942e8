"""Segment-integrated projection (AL_PROJ_INTEGRATED, the variant Sec. 6
proposes) on the GPU against the FP64 oracle: random instances of both
precisions (first step: gathered), the canopy over two steps (the second
replays the segment pass's records), replay equal to gather bit for bit,
and instances of both projections in one batch equal to each alone."""
import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W
from paper_2609_39443_b300.al import OPT_RECORD, ST_REPLAYED

from helpers import BRICK_PASSES, compare, run_gpu

pytestmark = pytest.mark.gpu

KINDS = ("stem", "arc", "random", "flat", "point", "dup")


@pytest.mark.parametrize("case", [(81, "fp32", {}), (82, "fp64", dict(has_alpha=True)),
                                  (83, "fp32", dict(eps_cells=(0.6, 1.2))), (84, "fp32", dict(eps_cells=(2.5, 4.0)))],
                         ids=["81", "82", "83", "84"])
def test_integrated_random_instances(case):
    seed, prec, extra = case
    wl = W.with_projection(W.make_random(seed, 36, 30, 26, n_lines=8, precision=prec, kinds=KINDS, **extra),
                           "integrated")
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label=f"integrated {seed}", sumF_ref="abs")
    for k in (0, 1, 2, 3, 4, 5):
        assert g["status"][k] == o["status"][k], (k, g["status"], o["status"])
    print("integrated", seed, m)


def _steps(wl, n, record):
    import torch
    from paper_2609_39443_b300.al import Instance
    inst = Instance(wl)
    inst.grid.set_option(OPT_RECORD, 1 if record else 2)
    out = []
    for _ in range(n):
        inst.status.zero_()
        inst.step()
        torch.cuda.synchronize()
        out.append({"S": inst.S.cpu().numpy().copy(), "F": inst.F[:, :wl.beams.n_points].cpu().numpy().copy(),
                    "totals": inst.totals.cpu().numpy().copy(), "status": inst.status.cpu().numpy().copy()})
    inst.close()
    return out


def test_integrated_canopy_replayed_matches_the_oracle():
    wl = W.with_projection(W.make_canopy(7, 2.0), "integrated")
    out = _steps(wl, 2, True)
    o1 = oracle.point_step(wl.grid, wl.beams, wl.step)
    o2 = oracle.sample_drag_spread(wl, f_prev=o1["f"])
    g = {k: out[1][k].astype(np.float64) if k in ("S", "F") else out[1][k] for k in out[1]}
    m = compare(wl, g, o2, label="integrated canopy")
    assert out[1]["status"][ST_REPLAYED] > 0
    print("integrated canopy", m)


@pytest.mark.parametrize("name", ["canopy", "random_fp64"])
def test_integrated_replay_equals_gather_bitwise(name):
    if name == "canopy":
        wl = W.make_canopy(8, 2.0, nx=128, ny=96, nz=96, n_sx=8, n_sy=6, n_cv=60, height=0.3)
    else:
        wl = W.make_random(85, 40, 33, 30, n_lines=8, precision="fp64", kinds=("stem", "arc", "random"))
    wl = W.with_projection(wl, "integrated")
    on, off = _steps(wl, 3, True), _steps(wl, 3, False)
    for k in range(3):
        for key in ("S", "F", "totals"):
            np.testing.assert_array_equal(on[k][key], off[k][key], err_msg=key)
    assert on[2]["status"][ST_REPLAYED] > 0


def test_integrated_batch_equals_alone():
    import torch
    from paper_2609_39443_b300.al import Batch, Instance
    wls = W.make_batched(9, 4, max_cells=96 * 64 * 64)
    wls = [W.with_projection(w, "integrated") if q % 2 == 0 else w for q, w in enumerate(wls)]
    alone, inb = [Instance(w, options=BRICK_PASSES) for w in wls], [Instance(w) for w in wls]
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
    batch.close()
    for x in alone + inb:
        x.close()
