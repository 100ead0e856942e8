"""al_line_forces_noalloc, the entry point for callers that cannot allocate
device memory (it keeps its line table in a fixed __device__ array instead),
against the line forces of al_sample_drag_spread on the same inputs, within
the tolerance the parity tests use for F, on two calls in a row (the second
relaxed against a previous force).  Collected last on purpose."""
import numpy as np
import pytest

from paper_2609_39443_b300 import workloads as W

from helpers import TOL_SUMF_FP32

pytestmark = pytest.mark.gpu


def test_noalloc_line_forces_match_the_step_on_two_calls():
    import torch
    from paper_2609_39443_b300.al import Instance, line_forces_noalloc

    tol = 10 * TOL_SUMF_FP32            # per-point F tolerance of the parity tests
    w1 = W.make_canopy(4, 2.0)
    w2 = W.make_random(41, 36, 30, 28, n_lines=12, kinds=("stem", "arc", "random", "point"), has_alpha=True)

    # call 1: un-relaxed forces, compared with the first step of an instance
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

    for ref, F, wl in ((ref1, F1, w1), (ref2, F2, w2)):
        a = ref.F[:, :wl.beams.n_points].double().cpu().numpy()
        b = F[:, :wl.beams.n_points].double().cpu().numpy()
        err = np.abs(a - b).max() / np.abs(a).max()
        assert err <= tol, (wl.name, err)
    # the point counters agree with the step's
    s_ref = ref1.status.cpu().numpy()
    s_new = st1.cpu().numpy()
    for k in (0, 1, 2, 3):
        assert s_ref[k] == s_new[k]
    ref1.close()
    ref2.close()


def test_noalloc_rejects_oversized_inputs():
    import torch
    from paper_2609_39443_b300.al import ALError, line_forces_noalloc
    wl = W.make_flume(0, nx=64, ny=64, nz=32, n_sx=40, n_sy=40, n_cv=50, height=0.1)   # 80000 points
    U = torch.zeros((3, wl.grid.n_cells), dtype=torch.float32, device="cuda")
    P = torch.zeros((3, wl.beams.n_points), dtype=torch.float32, device="cuda")
    F = torch.zeros_like(P)
    with pytest.raises(ALError):
        line_forces_noalloc(wl.grid, wl.beams, U, P, P, F, alpha=U[0])
