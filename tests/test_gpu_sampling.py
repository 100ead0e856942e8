"""Sampling operators on the GPU against the FP64 oracle: the kernel-weighted
volume average (sampling mode 2, one warp per actuator point) on random
instances of both precisions, on a kernel narrower than a cell (where some
points have no cell centre inside the support and take the containing
cell), on the full-size canopy, on the flume with its two-phase density and
sampling plane, together with the inertia term, and inside a batch next to
instances that sample trilinearly (bit for bit equal to each alone)."""
import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W

from helpers import BRICK_PASSES, compare, run_gpu

pytestmark = pytest.mark.gpu

KINDS = ("stem", "arc", "random", "flat", "point", "dup")

GAUSS_CASES = [
    # (seed, nx, ny, nz, precision, extra)
    (61, 37, 29, 21, "fp32", {}),
    (62, 40, 33, 19, "fp64", dict(has_alpha=True)),
    (63, 31, 31, 31, "fp32", dict(drag_mode=W.DRAG_SPLIT, has_alpha=True, n_p=(0.0, 1.0, 0.0))),
    (64, 23, 19, 17, "fp32", dict(eps_cells=(0.12, 0.3))),
    (65, 22, 20, 18, "fp64", dict(eps_cells=(0.12, 0.3))),
    (66, 64, 48, 40, "fp32", dict(eps_cells=(2.5, 4.0))),
]


@pytest.mark.parametrize("case", GAUSS_CASES, ids=[str(c[0]) for c in GAUSS_CASES])
def test_volume_average_random_instances(case):
    seed, nx, ny, nz, prec, extra = case
    wl = W.make_random(seed, nx, ny, nz, n_lines=8, precision=prec, kinds=KINDS,
                       sample_mode=W.SAMPLE_GAUSS, **extra)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label=f"gauss random {seed}", sumF_ref="abs")
    for k in (0, 1, 2, 3, 4, 5):
        assert g["status"][k] == o["status"][k], (k, g["status"], o["status"])
    print("gauss random", seed, m, g["status"][:8])


def test_volume_average_canopy_full_size():
    wl = W.with_sample_mode(W.make_canopy(0, 2.0), "gauss")
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label="gauss canopy")
    assert g["status"][:2].sum() == 0
    print("gauss canopy", m, "refined", g["status"][6])


def test_volume_average_flume_reduced():
    wl = W.with_sample_mode(W.make_flume(1, nx=256, ny=64, nz=128, n_sx=20, n_sy=8), "gauss")
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label="gauss flume reduced")
    print("gauss flume reduced", m)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_volume_average_with_inertia(prec):
    wl = W.with_inertia(W.make_random(67, 40, 34, 30, n_lines=8, precision=prec, has_alpha=True, kinds=KINDS,
                                      sample_mode=W.SAMPLE_GAUSS), 7)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label=f"gauss inertia {prec}", sumF_ref="abs")
    print("gauss inertia", prec, m)


def test_volume_average_differs_from_trilinear():
    """The operator really changes: the same instance sampled trilinearly and
    by volume average gives different forces (the oracle says by how much,
    and the GPU agrees with it in both modes)."""
    wl0 = W.make_random(68, 30, 28, 26, n_lines=6, kinds=("stem", "arc"))
    wl2 = W.with_sample_mode(wl0, "gauss")
    g0, g2 = run_gpu(wl0), run_gpu(wl2)
    o0, o2 = oracle.point_step(wl0.grid, wl0.beams, wl0.step), oracle.point_step(wl2.grid, wl2.beams, wl2.step)
    scale = np.abs(o0["F"]).max()
    gap = np.abs(o2["F"] - o0["F"]).max() / scale
    assert gap > 1e-3
    assert np.abs(g0["F"] - o0["F"]).max() / scale < 1e-5
    assert np.abs(g2["F"] - o2["F"]).max() / scale < 1e-5


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_with_volume_average_equals_alone(use_graph):
    import torch
    from paper_2609_39443_b300.al import Batch, Instance
    wls = W.make_batched(5, 4, max_cells=96 * 64 * 64)
    wls = [W.with_sample_mode(w, "gauss") if q % 2 == 0 else w for q, w in enumerate(wls)]
    alone = [Instance(w, options=BRICK_PASSES) for w in wls]
    inb = [Instance(w) for w in wls]
    batch = Batch(inb, use_graph=use_graph)
    for _ in range(2):
        for a in alone:
            a.status.zero_()
            a.step()
        for b in inb:
            b.status.zero_()
        batch.run()
        torch.cuda.synchronize()
        for a, b in zip(alone, inb):
            for x, y in ((a.S, b.S), (a.F, b.F), (a.totals, b.totals), (a.status, b.status)):
                np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    batch.close()
    for x in alone + inb:
        x.close()
