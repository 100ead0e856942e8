"""Quasi-static reconstruction of the beam side on the GPU
(al_beam_quasistatic) against the FP64 oracle: the kernel alone on the
forces of a step, in both precisions, and a coupled loop in which each
step's forces bend the stems and the next step samples and projects at the
bent positions."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W

from helpers import compare, run_gpu

pytestmark = pytest.mark.gpu

AXIS = (0.0, 0.0, 1.0)


def _EI(wl, value=2e-3):
    return np.full(wl.beams.n_lines, value) * (1.0 + 0.5 * np.arange(wl.beams.n_lines) / max(wl.beams.n_lines, 1))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_quasistatic_kernel_matches_the_oracle(prec):
    import torch
    from paper_2609_39443_b300.al import Instance
    wl = W.make_random(91, 36, 30, 40, n_lines=6, precision=prec, kinds=("stem", "arc", "random", "point"))
    inst = Instance(wl)
    inst.step()
    out = torch.empty_like(inst.P)
    EI = _EI(wl)
    inst.grid.beam_quasistatic(EI, AXIS, inst.P, inst.F, out)
    torch.cuda.synchronize()
    F = inst.F[:, :wl.beams.n_points].double().cpu().numpy()
    ref = oracle.beam_quasistatic(wl.beams, EI, AXIS, wl.step.P.astype(np.float64), F)
    got = out.double().cpu().numpy()
    disp = np.abs(ref - wl.step.P.astype(np.float64)).max()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.abs(got - ref).max() <= tol * max(disp, 1e-30) + (0 if prec == "fp64" else 1e-7 * np.abs(ref).max())
    inst.close()


def test_coupled_loop_with_the_quasistatic_beam():
    """Two coupled steps on the canopy: the first step's forces bend the
    stems, the second samples and projects at the bent positions."""
    import torch
    from paper_2609_39443_b300.al import Instance
    wl = W.make_canopy(11, 2.0, nx=128, ny=96, nz=96, n_sx=8, n_sy=6, n_cv=60, height=0.3)
    EI = _EI(wl, 5e-3)
    inst = Instance(wl)
    inst.step()
    P1 = torch.empty_like(inst.P)
    inst.grid.beam_quasistatic(EI, AXIS, inst.P, inst.F, P1)
    inst.P.copy_(P1)
    inst.status.zero_()
    inst.step()
    torch.cuda.synchronize()
    g = {"S": inst.S.double().cpu().numpy(), "F": inst.F[:, :wl.beams.n_points].double().cpu().numpy(),
         "totals": inst.totals.cpu().numpy(), "status": inst.status.cpu().numpy()}
    # the same loop in the oracle, the bent positions rounded to the field precision as on the GPU
    o1 = oracle.point_step(wl.grid, wl.beams, wl.step)
    P1o = oracle.beam_quasistatic(wl.beams, EI, AXIS, wl.step.P.astype(np.float64), o1["F"])
    moved = np.abs(P1o - wl.step.P).max() / wl.grid.h
    assert moved > 0.05, moved                    # the stems really bend (in cells)
    P1g = P1.double().cpu().numpy()
    assert np.abs(P1g - P1o).max() < 1e-5 * wl.grid.h * 10
    wl2 = replace(wl, step=replace(wl.step, P=P1g.astype(wl.step.P.dtype)))
    o2 = oracle.sample_drag_spread(wl2, f_prev=o1["f"])
    m = compare(wl2, g, o2, label="coupled canopy")
    print("coupled canopy", m, "max bend (cells)", moved)
    inst.close()
