"""Continuous batching in the library (al_server_*): simulations served in
a mix of waves (with admission by device bytes forcing some to wait for
others to leave) produce, step for step, the same line forces and final
momentum source as each simulation run alone, bit for bit; and what the
server admits is what the device gives up (cudaMemGetInfo)."""
import numpy as np
import pytest

from paper_2609_39443_b300 import workloads as W
from paper_2609_39443_b300.serve import BatchServer, Sim, instance_footprint, poisson_arrivals

from helpers import BRICK_PASSES

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("reflect", [False, True], ids=["truncated", "reflected-bed"])
def test_served_mix_equals_each_simulation_alone(reflect):
    import torch
    from paper_2609_39443_b300.al import Instance
    wls = W.make_batched(31, 6, max_cells=64 * 48 * 40)
    if reflect:                     # every other simulation reflects its kernel at the bed
        wls = [W.with_reflect(w, W.REFLECT_Z_LO) if i % 2 == 0 else w for i, w in enumerate(wls)]
    sims = [Sim(w, 3) for w in wls]
    need = [s.buffer_bytes() + instance_footprint(s) for s in sims]
    budget = int(2.5 * max(need))                             # two or three resident at a time
    arr = poisson_arrivals(sims, 5000.0, seed=11)
    srv = BatchServer(sims, budget, n_slots=4, record=True)
    st = srv.run(arr)
    assert st.completed == len(arr)
    assert st.peak_mem <= budget
    for s, sim in enumerate(sims):
        inst = Instance(sim.wl, options=BRICK_PASSES)
        for k in range(sim.n_steps):
            inst.set_points(P=sim.positions(k))
            inst.step()
            torch.cuda.synchronize()
            F = inst.F[:, :sim.wl.beams.n_points].cpu().numpy()
            np.testing.assert_array_equal(F, srv.results[(s, k)])
        np.testing.assert_array_equal(inst.S.cpu().numpy(), srv.final_S[s])
        inst.close()


def test_admitted_memory_stays_within_the_budget():
    """Admit simulations through the C ABI until the server refuses: the
    device memory they took (library instances and the caller's buffers, by
    cudaMemGetInfo) is what the server counts, up to page rounding, and
    stays within the budget."""
    import torch
    from paper_2609_39443_b300.al import Server
    from paper_2609_39443_b300.serve import CudaBackend
    wls = W.make_batched(41, 8, max_cells=96 * 64 * 64)
    sims = [Sim(w, 1) for w in wls]
    need = [s.buffer_bytes() + instance_footprint(s) for s in sims]
    budget = int(sum(sorted(need)[:5]) + 1)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0 = torch.cuda.mem_get_info()[0]
    srv = Server(budget, 8, 8, max(s.n_points for s in sims), "fp32")
    be = CudaBackend()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]             # the server's own staging
    keep, admitted = [], 0
    for s in sims:
        b = be.buffers(s)
        q = srv.admit(s.wl.grid, s.wl.beams, b.sin, b.sout, b.nbytes)
        if q is None:
            del b
            continue
        keep.append(b)
        admitted += 1
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free2 = torch.cuda.mem_get_info()[0]
    used, resident = srv.footprint()
    assert resident == admitted >= 2
    assert used <= budget
    taken = free1 - free2
    assert taken <= budget, (taken, budget)
    # the server never counts less than the device gives up; it counts at
    # most a page of rounding more per allocation (three per simulation: the
    # library's two slabs and the caller's buffers; small slabs share pages)
    assert taken <= used + 2 * 2 ** 20, (taken, used)
    assert used - taken <= 3 * 2 * 2 ** 20 * resident, (taken, used)
    srv.close()
    del keep
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 8 * 2 ** 20     # everything returned


def test_a_wait_that_runs_out_returns_timeout_and_the_step_completes_later():
    """A server wait bounded at 0 s returns AL_ERR_TIMEOUT while the wave
    (a full canopy step, far longer than the launch) is still running; the
    request stays in flight, a later poll with the default limit retires it,
    and its forces are those of the same step run alone.  No GPU wait is
    left unbounded and nothing is made to fault."""
    import ctypes as C
    import torch
    from paper_2609_39443_b300.al import AL_ERR_ARG, AL_ERR_TIMEOUT, ALError, Instance, Server, lib
    from paper_2609_39443_b300.serve import CudaBackend
    wl = W.make_canopy(0)
    sim = Sim(wl, 1)
    be = CudaBackend()
    srv = Server(sim.buffer_bytes() + instance_footprint(sim) + (1 << 30), 1, 1, sim.n_points, "fp32")
    b = be.buffers(sim)
    q = srv.admit(wl.grid, wl.beams, b.sin, b.sout, b.nbytes)
    assert q is not None
    with pytest.raises(ALError):
        srv.set_timeout(-1.0)
    assert lib().al_server_set_timeout(srv.h, float("nan")) == AL_ERR_ARG
    srv.set_timeout(0.0)
    P = sim.positions(0)
    F = np.empty_like(P)
    srv.submit(q, P, F, 7)
    n = C.c_int(-1)
    rc = lib().al_server_poll(srv.h, srv._done, len(srv._done), C.byref(n), 1)   # launches, waits 0 s
    assert rc == AL_ERR_TIMEOUT and n.value == 0
    srv.set_timeout(10.0)
    tags = srv.poll(wait=True)
    while not tags:
        tags = srv.poll(wait=True)
    assert tags == [7]
    srv.release(q)
    srv.close()
    inst = Instance(wl, options=BRICK_PASSES)
    inst.set_points(P=P)
    inst.step()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(inst.F[:, :sim.n_points].cpu().numpy(), F)
    inst.close()
