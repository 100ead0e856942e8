"""Kernel reflected at grid faces (al_beam_desc.wall_reflect, the one-sided
kernel Sec. 6 proposes, read as a mirror) on the GPU against the FP64
oracle: lines against faces, edges and corners in both precisions, the
plain cantilever and a small canopy rooted on a reflecting bed, no change
for lines out of reach of the reflecting faces, and reflected instances
in a batch equal to each alone."""
import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W
from paper_2609_39443_b300.al import (OPT_RECORD, OPT_WEIGHTS, ST_SUPPORT, WEIGHTS_BRICK, ALError, Batch,
                                      Instance)

from helpers import BRICK_PASSES, compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", [(5, "fp64", 63), (6, "fp32", 63), (7, "fp32", 16 | 2), (8, "fp64", 4 | 32)],
                         ids=["all-fp64", "all-fp32", "bed-xhi-fp32", "ylo-zhi-fp64"])
def test_reflected_walls_match_the_oracle(case):
    seed, prec, mask = case
    wl = W.with_reflect(W.make_walls(seed, precision=prec), mask)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label=f"walls {seed} mask {mask}")
    for k in range(6):
        assert g["status"][k] == o["status"][k], (k, g["status"], o["status"])
    assert g["status"][ST_SUPPORT] == oracle.count_support(wl.grid, wl.beams, wl.step.P)
    # the reflection moved mass: the plain kernel differs near the faces
    plain = oracle.sample_drag_spread(W.with_reflect(wl, 0))
    assert np.abs(plain["S"] - o["S"]).max() > 1e-3 * np.abs(o["S"]).max()
    print("walls", seed, mask, m)


def test_reflected_bed_plain_cantilever():
    wl = W.with_reflect(W.make_plain(3), W.REFLECT_Z_LO)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    compare(wl, g, o, label="plain reflected bed")


def test_reflected_bed_small_canopy_two_steps():
    wl = W.with_reflect(W.make_canopy(2, 2.0, nx=64, ny=48, nz=64, n_sx=4, n_sy=4, n_cv=30, height=0.15),
                        W.REFLECT_Z_LO)
    g = run_gpu(wl, steps=2)
    o1 = oracle.point_step(wl.grid, wl.beams, wl.step)
    o2 = oracle.sample_drag_spread(wl, f_prev=o1["f"])
    compare(wl, g, o2, label="canopy reflected bed")


def test_faces_out_of_reach_change_nothing():
    """The canopy's stems are far from the x+ and y- faces: reflecting them
    gives the same bits as the same passes without reflection."""
    import torch
    wl = W.make_canopy(3, 2.0, nx=96, ny=64, nz=48, n_sx=3, n_sy=3, n_cv=20, height=0.1)
    outs = []
    for mask in (0, W.REFLECT_X_HI | W.REFLECT_Y_LO):
        inst = Instance(W.with_reflect(wl, mask), options=BRICK_PASSES)
        inst.grid.set_option(OPT_WEIGHTS, WEIGHTS_BRICK)
        inst.grid.set_option(OPT_RECORD, 0)
        outs.append(run_gpu(wl, inst=inst))
        inst.close()
    for k in ("S", "F", "totals"):
        np.testing.assert_array_equal(outs[0][k], outs[1][k], err_msg=k)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_with_reflected_instances_equals_alone(use_graph):
    """Reflected and plain instances in one batch: each gives the bits it
    gives alone (the reflected ones run in their own batched kernels)."""
    import torch
    wls = [W.with_reflect(W.make_walls(11), 63), W.make_walls(12),
           W.with_reflect(W.make_canopy(4, 2.0, nx=64, ny=48, nz=64, n_sx=3, n_sy=3, n_cv=24, height=0.12),
                          W.REFLECT_Z_LO)]
    alone = [Instance(w, options=BRICK_PASSES) for w in wls]
    inb = [Instance(w) for w in wls]
    batch = Batch(inb, use_graph=use_graph)
    try:
        for _ in range(2):
            for a in alone:
                a.status.zero_()
                a.step()
            for x in inb:
                x.status.zero_()
            batch.run()
            torch.cuda.synchronize()
            for w, a, x in zip(wls, alone, inb):
                for k in ("S", "F", "totals", "status"):
                    np.testing.assert_array_equal(getattr(a, k).cpu().numpy(), getattr(x, k).cpu().numpy(),
                                                  err_msg=f"{w.name} {k}")
    finally:
        batch.close()
        for x in alone + inb:
            x.close()


@pytest.mark.parametrize("bad", ["integrated", "mask", "too_deep"])
def test_reflection_arguments_are_checked(bad):
    wl = W.make_walls(2)
    if bad == "integrated":
        wl = W.with_reflect(W.with_projection(wl, "integrated"), 16)
    elif bad == "mask":
        wl = W.with_reflect(wl, 64)
    else:                           # 3 eps / h = 4.5 + 1 ghost layers > the 4 cells along x
        wl = W.with_reflect(W.make_random(9, 4, 12, 12, n_lines=1, eps_cells=(1.5, 1.5), kinds=("stem",)), 1)
    with pytest.raises(ALError):
        Instance(wl)


def test_reflection_from_both_faces_of_a_narrow_grid():
    """A grid only a few kernel widths across: cells near both faces of an
    axis take images across each (three choices per axis, up to 26 images
    at once), with ghosts as deep as the grid allows."""
    from paper_2609_39443_b300.workloads import GridSpec, StepInput, Workload, _beams_from_lines
    h = 0.01
    g = GridSpec(10, 9, 8, h, precision="fp64", rho_const=1000.0)
    rng = np.random.default_rng(3)
    t = np.linspace(0.0, 1.0, 7)
    lines = [np.stack([h * (2.0 + 5.0 * t), h * (4.5 + 0.5 * np.sin(4 * t)), h * (1.0 + 6.0 * t)]),
             np.stack([h * (8.5 - 2.0 * t), h * (1.0 + 7.0 * t), np.full_like(t, 4.2 * h)])]
    U = rng.normal(0.0, 0.05, size=(3, g.n_cells))
    U[0] += 0.2
    P = np.concatenate(lines, axis=1)
    beams = _beams_from_lines(lines, [np.full(7, h), np.full(7, h)], d=0.004, cdn=1.2, cdt=0.01, eps=1.5 * h,
                              ell_s=0.5 * h)
    wl = W.with_reflect(Workload("narrow", g, beams, StepInput(U=U, P=P, Pdot=rng.normal(0, 0.01, P.shape))), 63)
    g_out, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    compare(wl, g_out, o, label="narrow grid, all faces")
    assert g_out["status"][ST_SUPPORT] == oracle.count_support(wl.grid, wl.beams, wl.step.P)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_reflection_with_volume_average_and_inertia(prec):
    """The variants compose: the Gaussian volume-average sampler and the
    inertia term at the points, the kernel reflected at every face in the
    projection."""
    wl = W.with_reflect(W.with_sample_mode(W.with_inertia(W.make_walls(13, precision=prec), 14), "gauss"), 63)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    compare(wl, g, o, label=f"walls gauss inertia reflected {prec}")


def test_reflected_bed_full_canopy():
    """The full canopy (256x128x128, 400 stems) with a reflecting bed, in the
    options the bench uses for it, against the oracle."""
    wl = W.with_reflect(W.make_canopy(0, 2.0), W.REFLECT_Z_LO)
    inst = Instance(wl)
    inst.autotune()
    g = run_gpu(wl, inst=inst)
    inst.close()
    o = oracle.sample_drag_spread(wl)
    compare(wl, g, o, label="canopy reflected bed")
    assert g["status"][ST_SUPPORT] == oracle.count_support(wl.grid, wl.beams, wl.step.P)
