"""al_line_forces_noalloc, the entry point for callers that cannot allocate
device memory where they need the line forces (an allocator that forbids
allocation after start-up, a plug-in whose host owns all device memory): it
keeps its line table in a fixed __device__ array instead.  Its forces are
checked against those of al_sample_drag_spread on the same inputs and
against the FP64 oracle, within the per-point F tolerance of the parity
tests, on two calls in a row (the second relaxed against a previous force),
with the inertia term, and on an empty line set.  Collected last on purpose:
a failure here comes after every other test has run."""
import ctypes as C
from dataclasses import replace

import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W

from helpers import TOL_SUMF_FP32

pytestmark = pytest.mark.gpu

TOL_F = 10 * TOL_SUMF_FP32            # per-point F tolerance of the parity tests


def _err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _np(F, n):
    return F[:, :n].double().cpu().numpy()


def test_noalloc_line_forces_match_the_step_and_the_oracle_on_two_calls():
    import torch
    from paper_2609_39443_b300.al import Instance, line_forces_noalloc

    w1 = W.make_canopy(4, 2.0)
    w2 = W.make_random(41, 36, 30, 28, n_lines=12, kinds=("stem", "arc", "random", "point"), has_alpha=True)

    # call 1: un-relaxed forces, against the first step of an instance
    ref1 = Instance(w1)
    ref1.step()
    F1 = torch.empty_like(ref1.F)
    st1 = torch.zeros(16, dtype=torch.int32, device="cuda")
    line_forces_noalloc(w1.grid, w1.beams, ref1.U, ref1.P, ref1.Pdot, F1, status=st1)

    # call 2: relaxed against the previous force of a second instance
    ref2 = Instance(w2)
    ref2.step()
    f_prev = torch.empty((3, w2.beams.n_points), dtype=ref2.dtype, device="cuda")
    assert ref2.grid.get_state(f_prev)
    ref2.status.zero_()
    ref2.step()
    F2 = torch.empty_like(ref2.F)
    line_forces_noalloc(w2.grid, w2.beams, ref2.U, ref2.P, ref2.Pdot, F2, alpha=ref2.alpha, f_prev=f_prev)
    torch.cuda.synchronize()

    # the oracle's own two steps
    o1 = oracle.point_step(w1.grid, w1.beams, w1.step)
    o2a = oracle.point_step(w2.grid, w2.beams, w2.step)
    o2 = oracle.point_step(w2.grid, w2.beams, w2.step, f_prev=o2a["f"])

    n1, n2 = w1.beams.n_points, w2.beams.n_points
    assert _err(_np(F1, n1), _np(ref1.F, n1)) <= TOL_F
    assert _err(_np(F2, n2), _np(ref2.F, n2)) <= TOL_F
    assert _err(_np(F1, n1), o1["F"]) <= TOL_F
    assert _err(_np(F2, n2), o2["F"]) <= TOL_F
    # the point counters agree with the step's and the oracle's
    s_ref = ref1.status.cpu().numpy()
    s_new = st1.cpu().numpy()
    for k in (0, 1, 2, 3):
        assert s_ref[k] == s_new[k] == o1["status"][k]
    # later calls take no device memory: the free bytes do not move
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        line_forces_noalloc(w2.grid, w2.beams, ref2.U, ref2.P, ref2.Pdot, F2, alpha=ref2.alpha, f_prev=f_prev)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref1.close()
    ref2.close()


def test_noalloc_inertia_term():
    import torch
    from paper_2609_39443_b300.al import Instance, line_forces_noalloc

    wl = W.with_inertia(W.make_random(43, 32, 30, 26, n_lines=8, kinds=("stem", "arc"), has_alpha=True), 7)
    ref = Instance(wl)
    ref.step()
    F = torch.empty_like(ref.F)
    line_forces_noalloc(wl.grid, wl.beams, ref.U, ref.P, ref.Pdot, F, alpha=ref.alpha,
                        U_prev=ref.U_prev, Pddot=ref.Pddot, dt=wl.step.dt)
    torch.cuda.synchronize()
    n = wl.beams.n_points
    o = oracle.point_step(wl.grid, wl.beams, wl.step)
    assert _err(_np(F, n), _np(ref.F, n)) <= TOL_F
    assert _err(_np(F, n), o["F"]) <= TOL_F
    # the term matters here: the drag-only forces differ by far more
    drag = oracle.point_step(wl.grid, replace(wl.beams, cm_n=None, cm_t=None), wl.step)
    assert _err(drag["F"], o["F"]) > 100 * TOL_F
    ref.close()


def test_noalloc_empty_line_set():
    import torch
    from paper_2609_39443_b300 import al

    wl = W.make_random(44, 16, 16, 16, n_lines=2, kinds=("stem",))
    g = wl.grid
    gd = al.GridDesc(g.nx, g.ny, g.nz, g.h, (C.c_double * 3)(*g.origin), al.AL_FP32, 0, g.rho1, g.rho2,
                     g.rho_const)
    bd = al.BeamDesc()                      # n_lines = 0, every array NULL
    bd.tau = 1e-6
    U = torch.zeros((3, g.n_cells), dtype=torch.float32, device="cuda")
    sin, _ = al.step_descriptors(U, None, None, U, None)
    fo = (C.c_void_p * 3)(None, None, None)
    st = torch.full((16,), 5, dtype=torch.int32, device="cuda")
    stream = al._stream_ptr(None)
    rc = al.lib().al_line_forces_noalloc(C.byref(gd), C.byref(bd), C.byref(sin), None, fo,
                                         C.cast(st.data_ptr(), C.POINTER(C.c_int)), stream)
    assert rc == al.AL_OK
    rc = al.lib().al_line_forces_noalloc(C.byref(gd), C.byref(bd), C.byref(sin), None, fo, None, stream)
    assert rc == al.AL_OK
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 5).all()    # nothing counted into the caller's array


def test_noalloc_rejects_oversized_and_unsupported_inputs():
    import torch
    from paper_2609_39443_b300.al import ALError, line_forces_noalloc
    wl = W.make_flume(0, nx=64, ny=64, nz=32, n_sx=40, n_sy=40, n_cv=50, height=0.1)   # 80000 points
    U = torch.zeros((3, wl.grid.n_cells), dtype=torch.float32, device="cuda")
    P = torch.zeros((3, wl.beams.n_points), dtype=torch.float32, device="cuda")
    F = torch.zeros_like(P)
    with pytest.raises(ALError, match="capacity"):
        line_forces_noalloc(wl.grid, wl.beams, U, P, P, F, alpha=U[0])
    small = W.with_sample_mode(W.make_random(45, 16, 16, 16, n_lines=2, kinds=("stem",)), "gauss")
    U = torch.zeros((3, small.grid.n_cells), dtype=torch.float32, device="cuda")
    P = torch.zeros((3, small.beams.n_points), dtype=torch.float32, device="cuda")
    with pytest.raises(ALError, match="invalid argument"):
        line_forces_noalloc(small.grid, small.beams, U, P, P, torch.zeros_like(P))
