"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several 16x16x8 bricks and ragged tails; the canopy runs at its
full size, the flume at a reduced and at its full size.  Tolerances
(tests/helpers.py): S within 1e-5 of max|S| for FP32 instances, total
force within 1e-6, conservation of the resultant within 1e-6 (FP64
instances: 1e-11 / 1e-12 / 1e-12).
"""
import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W
from paper_2609_39443_b300.workloads import BeamSpec, GridSpec, StepInput, Workload

from helpers import compare, run_gpu

pytestmark = pytest.mark.gpu


def test_plain_fp64():
    wl = W.make_plain(0)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label="plain")
    assert g["status"][:2].sum() == 0
    print("plain", m)


@pytest.mark.parametrize("eps_cells", [1.5, 2.0, 3.0])
def test_canopy_full_size(eps_cells):
    wl = W.make_canopy(0, eps_cells)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label=f"canopy eps={eps_cells}")
    assert g["status"][8] == oracle.count_support(wl.grid, wl.beams, wl.step.P)
    print("canopy", eps_cells, m, "refined", g["status"][6], "irregular", g["status"][7])


def test_flume_reduced():
    wl = W.make_flume(1, nx=256, ny=64, nz=128, n_sx=20, n_sy=8)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label="flume reduced")
    print("flume reduced", m)


def test_flume_full_size():
    wl = W.make_flume(0)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label="flume")
    print("flume", m, "refined", g["status"][6])


RANDOM_CASES = [
    # (seed, nx, ny, nz, precision, kinds, extra)
    (1, 37, 29, 21, "fp32", ("stem", "arc", "random", "flat", "point", "dup"), {}),
    (2, 40, 33, 19, "fp64", ("stem", "arc", "random", "flat", "point", "dup"), {}),
    (3, 23, 45, 17, "fp32", ("stem", "arc"), dict(sample_mode=W.SAMPLE_CELL)),
    (4, 31, 31, 31, "fp32", ("stem", "random"), dict(drag_mode=W.DRAG_SPLIT, has_alpha=True)),
    (5, 48, 20, 26, "fp32", ("stem", "flat"), dict(n_p=(0.0, 1.0, 0.0))),
    (6, 33, 17, 40, "fp64", ("arc", "random", "point"), dict(sample_mode=W.SAMPLE_CELL, has_alpha=True)),
    (7, 17, 17, 9, "fp32", ("stem", "arc", "random", "flat", "point", "dup"), dict(eps_cells=(0.6, 1.2))),
    (8, 64, 48, 40, "fp32", ("stem",), dict(eps_cells=(2.5, 4.0))),
]


@pytest.mark.parametrize("case", RANDOM_CASES, ids=[str(c[0]) for c in RANDOM_CASES])
def test_random_instances(case):
    seed, nx, ny, nz, prec, kinds, extra = case
    wl = W.make_random(seed, nx, ny, nz, n_lines=8, precision=prec, kinds=kinds, **extra)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label=f"random {seed}", sumF_ref="abs")
    # the device counters agree with the oracle's, and so does the number of
    # (cell, line) pairs inside the 3-eps support (every cut-off decision)
    for k in (0, 1, 2, 3, 4, 5):
        assert g["status"][k] == o["status"][k], (k, g["status"], o["status"])
    assert g["status"][8] == oracle.count_support(wl.grid, wl.beams, wl.step.P)
    print("random", seed, m, g["status"][:8])


def test_degenerate_grids():
    for dims in [(1, 1, 1), (1, 7, 9), (5, 1, 3), (40, 1, 1), (3, 50, 2)]:
        wl = W.make_random(20 + sum(dims), *dims, h=0.01, n_lines=3, kinds=("stem", "point", "flat"))
        g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
        compare(wl, g, o, label=f"grid {dims}", sumF_ref="abs")


def test_no_lines_writes_zeros():
    grid = GridSpec(20, 18, 10, 0.01)
    b = BeamSpec(line_off=np.zeros(1, np.int32), d=np.zeros(0), cdn=np.zeros(0), cdt=np.zeros(0),
                 eps=np.zeros(0), ell_s=np.zeros(0), alpha_f=np.zeros(0), cv_len=np.zeros(0))
    U = np.random.default_rng(0).normal(size=(3, grid.n_cells)).astype(np.float32)
    wl = Workload("empty", grid, b, StepInput(U=U, P=np.zeros((3, 0), np.float32), Pdot=np.zeros((3, 0), np.float32)))
    import torch
    from paper_2609_39443_b300.al import Instance
    inst = Instance(wl)
    inst.S.fill_(7.0)
    inst.step()
    torch.cuda.synchronize()
    assert float(inst.S.abs().max()) == 0.0
    assert np.all(inst.totals.cpu().numpy() == 0.0)
    inst.close()


def test_relaxation_over_two_steps():
    wl = W.make_random(30, 32, 30, 28, n_lines=6, kinds=("stem", "arc"))
    o1 = oracle.point_step(wl.grid, wl.beams, wl.step)
    o2 = oracle.sample_drag_spread(wl, f_prev=o1["f"])
    g2 = run_gpu(wl, steps=2)
    compare(wl, g2, o2, label="second step", sumF_ref="abs")


def test_deterministic_bitwise():
    wl = W.make_canopy(3, 2.0, nx=96, ny=64, nz=72, n_sx=6, n_sy=6, n_cv=40, height=0.2)
    a, b = run_gpu(wl), run_gpu(wl)
    np.testing.assert_array_equal(a["S"], b["S"])
    np.testing.assert_array_equal(a["F"], b["F"])
    np.testing.assert_array_equal(a["totals"], b["totals"])


def test_state_export_import():
    import torch
    from paper_2609_39443_b300.al import Instance
    wl = W.make_random(31, 30, 30, 30, n_lines=4, kinds=("stem",))
    i1 = Instance(wl)
    i1.step()
    fp = torch.empty((3, wl.beams.n_points), dtype=torch.float32, device="cuda")
    assert i1.grid.get_state(fp)
    i1.step()
    i2 = Instance(wl)
    i2.grid.set_state(fp, True)
    i2.step()
    torch.cuda.synchronize()
    assert torch.equal(i1.S, i2.S) and torch.equal(i1.F, i2.F)
    i1.close(); i2.close()


def test_projection_positions_and_tangents_given():
    wl = W.make_random(32, 36, 30, 26, n_lines=5, kinds=("stem", "arc", "flat"))
    rng = np.random.default_rng(1)
    Ps = (wl.step.P.astype(np.float64) + rng.normal(0, 0.3 * wl.grid.h, wl.step.P.shape)).astype(np.float32)
    T = rng.normal(size=wl.step.P.shape).astype(np.float32)
    wl.step.P_spread = Ps
    wl.step.tangent = T
    wl.beams.tangents_given = True
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    compare(wl, g, o, label="P_spread+tangent", sumF_ref="abs")


def test_zero_weight_nodes_deposit():
    grid = GridSpec(12, 12, 12, 1.0)
    P = np.array([[3.2, 5.7, 8.9], [4.1, 4.3, 6.6], [2.2, 6.9, 9.3]], np.float32)
    b = BeamSpec(line_off=np.array([0, 3], np.int32), d=np.array([0.01]), cdn=np.array([1.2]),
                 cdt=np.array([0.01]), eps=np.array([0.05]), ell_s=np.array([1.0]), alpha_f=np.array([1.0]),
                 cv_len=np.ones(3))
    U = np.zeros((3, grid.n_cells), np.float32)
    U[0] = 2.0
    wl = Workload("zw", grid, b, StepInput(U=U, P=P, Pdot=np.zeros_like(P)))
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    assert g["status"][4] == 3 and o["status"][4] == 3
    compare(wl, g, o, label="zero weight", sumF_ref="abs")


def test_dense_stems_several_batches_and_chunks():
    """More than 512 lines (several mask chunks per brick) and more than 32
    candidate lines per brick (several batches, S accumulated across them)."""
    wl = W.random_canopy(11, 64, 48, 32, 0.005, 700, 12, 2.0, name="dense")
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label="dense")
    assert g["status"][8] == oracle.count_support(wl.grid, wl.beams, wl.step.P)
    print("dense", m)


def test_fine_segments_zero_weight_deposits():
    """Segments a quarter of a cell long leave many nodes with w_k = 0; each
    deposits its load in the cell that contains it, inside the projection."""
    wl = W.random_canopy(12, 48, 40, 32, 0.005, 60, 64, 1.6, name="fine")
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    assert o["status"][4] > 0 and g["status"][4] == o["status"][4]
    m = compare(wl, g, o, label="fine")
    print("fine", m, "zero-weight nodes", o["status"][4])


@pytest.mark.parametrize("case", ["random-fp32", "random-fp64", "canopy"])
def test_inertia_term(case):
    """Morison inertia (added mass and Froude-Krylov, Eq. fext_addedmass) with
    a time-varying fluid and accelerating beams, against the oracle."""
    if case == "canopy":
        wl = W.with_inertia(W.make_canopy(2, 2.0), 6)
    else:
        prec = "fp64" if case.endswith("fp64") else "fp32"
        wl = W.with_inertia(W.make_random(51, 40, 34, 30, n_lines=8, precision=prec, has_alpha=True,
                                          kinds=("stem", "arc", "random", "flat", "point", "dup")), 5)
    g, o = run_gpu(wl), oracle.sample_drag_spread(wl)
    m = compare(wl, g, o, label=f"inertia {case}", sumF_ref="net" if case == "canopy" else "abs")
    print("inertia", case, m)
