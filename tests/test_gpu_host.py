"""al_step_host: the step with its fields and results in pinned host
memory, the copies on the caller's stream.  Alternating two streams and two
device buffer sets (the copies of one step overlapping the other's) gives
the results of the device-resident step bit for bit, over relaxed steps,
and they match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2609_39443_b300 import workloads as W

from helpers import compare

pytestmark = pytest.mark.gpu


def _host_inputs(inst):
    import torch
    h = {}
    for k in ("U", "P", "Pdot", "alpha", "P_spread", "tangent", "U_prev", "Pddot"):
        t = getattr(inst, k)
        h[k] = None if t is None else t.cpu().pin_memory()
    return h


@pytest.mark.parametrize("kind", ["flume", "random"])
def test_host_steps_on_two_streams_equal_the_device_steps(kind):
    import torch
    from paper_2609_39443_b300.al import Instance
    wl = (W.make_flume(5, nx=160, ny=48, nz=96, n_sx=14, n_sy=5, height=0.3) if kind == "flume"
          else W.make_random(23, 48, 40, 36, n_lines=8, kinds=("stem", "arc", "random"), has_alpha=True))
    ref = Instance(wl)
    for _ in range(3):
        ref.step()
    torch.cuda.synchronize()
    inst = Instance(wl)
    sets = [inst.own_buffers(), inst.buffers()]
    host_in = _host_inputs(inst)
    outs = [{"S": torch.empty(inst.S.shape, dtype=inst.S.dtype).pin_memory(),
             "F": torch.empty(inst.F.shape, dtype=inst.F.dtype).pin_memory()} for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k in range(3):
        inst.step_host({**host_in, **outs[k % 2]}, sets[k % 2], stream=streams[k % 2])
    torch.cuda.synchronize()
    last = outs[2 % 2]
    np.testing.assert_array_equal(last["S"].numpy(), ref.S.cpu().numpy())
    np.testing.assert_array_equal(last["F"].numpy(), ref.F.cpu().numpy())
    np.testing.assert_array_equal(inst.totals.cpu().numpy(), ref.totals.cpu().numpy())
    # and the oracle, relaxed twice against the previous forces
    o1 = oracle.point_step(wl.grid, wl.beams, wl.step)
    o2 = oracle.point_step(wl.grid, wl.beams, wl.step, f_prev=o1["f"])
    o3 = oracle.sample_drag_spread(wl, f_prev=o2["f"])
    g = {"S": last["S"].double().numpy(), "F": last["F"][:, :wl.beams.n_points].double().numpy(),
         "totals": inst.totals.cpu().numpy(), "status": inst.status.cpu().numpy()}
    compare(wl, g, o3, label=f"host steps {kind}")
    ref.close()
    inst.close()


def test_host_step_refuses_missing_descriptors():
    import ctypes as C
    from paper_2609_39443_b300.al import ALError, Instance, check, lib, step_descriptors
    wl = W.make_random(3, 24, 20, 16, n_lines=2)
    inst = Instance(wl)
    din, dout = step_descriptors(inst.U, inst.P, inst.Pdot, inst.S, inst.F, alpha=inst.alpha)
    with pytest.raises(ALError):
        check(lib().al_step_host(inst.grid.h, None, None, C.byref(din), C.byref(dout), None), "al_step_host")
    inst.close()
